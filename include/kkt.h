/*
 * kkt.h - C ABI of the GB300 solver for the heat-equation-constrained KKT system of
 * Cyr, "A 2-Level Domain Decomposition Preconditioner for KKT Systems with Heat-Equation
 * Constraints" (arXiv 2305.04421).
 *
 * Problem (Section 1, Eq 1; discretised in Section 2, Eqs 2-5): minimise
 *   1/2 int ||u - u~||^2 dt + omega/2 int ||z||^2 dt  subject to  u_t - nu Lap u = z,
 * on (0,Lx) x (0,Ly) with u = 0 on the boundary, u(0) = u_0, 5-point finite differences on
 * nx x ny intervals, backward Euler with Nt steps of dt = T/Nt. The optimality system is
 *   K (u, z, w) = (f_u, f_z, f),  K = [[M_u, 0, J^T], [0, omega M_z, L^T], [J, L, 0]]   (Eq 5)
 * with M_u = M_z = h I, h = dt dx dy, J block lower bidiagonal (diagonal I + dt nu A,
 * sub-diagonal -I) and L = -dt I.
 *
 * Vector layout (every double* below): a KKT vector is three blocks u | z | w, each of
 * V = Nt * (ny-1) * (nx-1) doubles ordered [n][j][i], n = 1..Nt the time node, j the y index,
 * i the x index (fastest). A "block" argument is one such V-vector.
 *
 * Pointers: unless an entry point says otherwise, vector pointers are DEVICE pointers (for
 * instance from torch CUDA tensors), contiguous, 8-byte aligned, owned by the caller; the
 * library never keeps them after the call returns. Input and output must not overlap unless
 * stated. `stream` is a cudaStream_t (NULL = the legacy default stream); the
 * asynchronous entry points only enqueue work on it.
 *
 * Errors: every int-returning entry point returns KKT_OK (0) on success, KKT_NOT_CONVERGED (1)
 * when a solve stopped at maxit, and a negative KKT_ERR_* code on failure; kkt_last_error()
 * then returns a message for the calling thread. A handle is not thread-safe: use one handle
 * per host thread and stream.
 */
#ifndef KKT_H
#define KKT_H

#ifdef __cplusplus
extern "C" {
#endif

enum kkt_status {
  KKT_OK = 0,
  KKT_NOT_CONVERGED = 1,
  KKT_ERR_INVALID_ARG = -1,
  KKT_ERR_OOM = -2,
  KKT_ERR_CUDA = -3,
  KKT_ERR_NONFINITE = -4,
  KKT_ERR_TIMEOUT = -5,
  KKT_ERR_BREAKDOWN = -6,
  KKT_ERR_UNSUPPORTED = -7
};

/* Arithmetic of the spatial transforms and time sweeps inside the preconditioner. */
enum kkt_precision {
  KKT_PREC_FP64 = 0,   /* FP64 everywhere */
  KKT_PREC_BF16 = 1,   /* DST GEMMs on tcgen05 tensor cores, BF16 in, FP32 accumulate; FP32 sweeps */
  KKT_PREC_TF32 = 2    /* as BF16 with TF32 operands */
};

/* Coarse level of the Schur-complement preconditioner (Section 3, Eqs 14-15). */
enum kkt_coarse {
  KKT_COARSE_EXACT = 0,    /* Nicolaides coarse space, exact coarse solve: the two-level method */
  KKT_COARSE_NONE = 1,     /* one-level RASQ (Eq 13) */
  KKT_COARSE_LEARNED = 2   /* learned correction on the lowest modes, exact solve elsewhere */
};

/* How the coarse correction is composed with RASQ (Eq 15). */
enum kkt_variant {
  KKT_MULTIPLICATIVE = 0,  /* x0 = R0^T S0^-1 R0 r ; y = x0 + S_RASQ^-1 (r - S-hat x0) */
  KKT_ADDITIVE = 1         /* y = R0^T S0^-1 R0 r + S_RASQ^-1 r */
};

/* Norm of the residual that FGMRES minimises and tests against tol. */
enum kkt_residual_norm {
  /* Discrete L2(0,T;L2) norms: the u and z rows (gradients of the objective) in the dual
   * norm, weight h^-1/2; the state-equation rows in the primal norm, weight h^1/2. */
  KKT_NORM_L2 = 0,
  /* Unweighted Euclidean norm over all three blocks. In FP64 its attainable relative value
   * is limited to about machine epsilon times |J| / h (about 3e-7 at 256 x 256, Nt = 1024). */
  KKT_NORM_EUCLIDEAN = 1
};

/* Orthogonalisation of the Arnoldi step. */
enum kkt_orth {
  /* modified Gram-Schmidt, one pass: for k = 0..j, h_kj = <q_k, w>, w -= h_kj q_k. Each step is
   * one streaming pass over q_k, q_k+1 and w (2 FP64 FMAs per element); GMRES with MGS is
   * backward stable (Paige, Rozloznik and Strakos, 2006). The oracle's orthogonalisation. */
  KKT_ORTH_MGS = 0,
  /* classical Gram-Schmidt with one conditional repeat (||w'||^2 < ||w||^2 / 2): all dots of a
   * pass in one multi-dot, one multi-axpy; 4 FMAs per element and basis vector when it repeats */
  KKT_ORTH_CGS2 = 1,
  /* MGS over pairs of basis vectors: both dots of a pair are taken on the same w, the pair is
   * subtracted in one pass that also takes the next pair's dots. 3 vector passes per basis
   * vector instead of 4, the same FMA count; equals MGS up to the pair's orthogonality error.
   * The default. */
  KKT_ORTH_MGS2 = 2,
  /* the same over blocks of four basis vectors (block MGS with the block's dots taken on one
   * w): 2.5 vector passes per basis vector, but each pass streams 9 vectors at once, which the
   * DRAM serves more slowly: no faster than pairs on GB300 */
  KKT_ORTH_MGS4 = 3,
  /* the same over blocks of eight: 2.25 vector passes per basis vector, 17 streams per pass */
  KKT_ORTH_MGS8 = 4
};

/* Local solves of the one-level part. */
enum kkt_local {
  /* RASQ (Eq 13): per subdomain (R_s Jhat R_s^T)^-T h (R_s Jhat R_s^T)^-1, the local problems
   * with zero initial and terminal conditions, as two sweeps */
  KKT_LOCAL_RASQ = 0,
  /* RAS (Eq 9): per subdomain the explicit local Schur complement (R_s S-hat R_s^T)^-1, a
   * tridiagonal solve in time per sine mode; an ablation that differs from RASQ only in the
   * first node's block (the zero initial condition) */
  KKT_LOCAL_RAS = 1
};

/* Basis the FGMRES iteration runs in. */
enum kkt_basis {
  /* grid values, as Eq 5 is written: every preconditioner apply does a forward and an inverse
   * 2D sine transform of the w block, every matvec is the 5-point stencil */
  KKT_BASIS_PHYSICAL = 0,
  /* sine-mode coefficients: f and x are transformed once (the orthonormal 2D DST-I of every
   * block, its own inverse), the iteration then runs without transforms (the preconditioner's
   * sweeps and coarse solve act per mode, the matvec's stencil becomes a product per mode), and
   * x is transformed back at exit. The transform is orthonormal and the residual weights are
   * per block, so inner products, norms and hence the iterates are those of the physical basis
   * in exact arithmetic. FP64 only. */
  KKT_BASIS_SPECTRAL = 1
};

/* Solver of the coarse problem S_0 c' = R_0 r (the operator after Eq 14). Per sine mode S_0 is
 * block tridiagonal in time: N_D blocks of 2 x 2, symmetric positive definite. Both solvers
 * are exact; they differ in how the work is spread over the GPU. */
enum kkt_coarse_solve {
  /* FP64: cyclic reduction when its per-configuration factors (19 doubles per block and mode,
   * about) take at most 256 MiB and one mode's system fits in shared memory, block Thomas
   * otherwise (measured: the factored cyclic solve is never slower; above the cap it gains
   * nothing measurable for its memory). BF16/TF32 (padded modes, no stored factors): cyclic
   * below 12288 spatial modes. */
  KKT_COARSE_SOLVE_AUTO = 0,
  /* block Thomas elimination, one thread per mode: R_0 r summed node by node, then N_D
   * dependent elimination steps and N_D back-substitution steps. The fewest FLOPs. */
  KKT_COARSE_SOLVE_THOMAS = 1,
  /* a multilevel hierarchy in time (the paper's conclusion names more levels as future work
   * without fixing them; this is its exact reading): block cyclic reduction. Level l+1 is the
   * exact Schur complement of level l onto every second of its blocks, again block
   * tridiagonal, down to one block after ceil(log2 N_D) levels, then back up. The subdomain
   * sums of R_0 r and each level's eliminations run in parallel over subdomains, so the
   * dependent chain is O(log N_D) instead of O(Nt). About three times Thomas's FLOPs.
   * Not used with the learned coarse correction (which falls back to Thomas). */
  KKT_COARSE_SOLVE_CYCLIC = 2
};

/* Owner of the time node shared by neighbouring subdomains (boolean partition of unity D_s). */
enum kkt_pou {
  KKT_POU_LEFT = 0,   /* the subdomain whose last step ends on the node */
  KKT_POU_RIGHT = 1   /* the subdomain whose first step starts from the node */
};

typedef struct kkt_options {
  int precision;    /* enum kkt_precision, default KKT_PREC_FP64 */
  int coarse;       /* enum kkt_coarse, default KKT_COARSE_EXACT */
  int variant;      /* enum kkt_variant, default KKT_MULTIPLICATIVE */
  int pou;          /* enum kkt_pou, default KKT_POU_LEFT */
  int restart;      /* FGMRES restart length, 1..32, default 30 */
  int jhat_sign;    /* -1 (default): Jhat = J - omega^-1/2 L; +1: the sign printed in Eq 7 */
  int residual_norm;  /* enum kkt_residual_norm, default KKT_NORM_L2 */
  int tc_split;     /* BF16 / TF32 only: 1 (default) every tensor-core transform uses hi + lo operands
                       (three products, FP32 accumulation); 0 single operands */
  int orth;         /* enum kkt_orth, default KKT_ORTH_MGS2 */
  int basis;        /* enum kkt_basis, default KKT_BASIS_PHYSICAL */
  int local;        /* enum kkt_local, default KKT_LOCAL_RASQ */
  double Lx, Ly;    /* domain (0,Lx) x (0,Ly), default 1, 1 */
  int coarse_solve; /* enum kkt_coarse_solve, default KKT_COARSE_SOLVE_AUTO */
} kkt_options;

typedef struct kkt_info {
  int nx, ny, Nt, n_sub;
  long long N;          /* (nx-1)(ny-1) spatial unknowns per time node */
  long long V;          /* N * Nt, unknowns per block */
  double dx, dy, dt, h; /* h = dt dx dy */
  long long workspace_bytes;  /* device memory the handle holds now */
} kkt_info;

#define KKT_HISTORY_MAX 1024
typedef struct kkt_stats {
  int iterations;          /* Arnoldi steps taken (one preconditioner apply + one matvec each) */
  int restarts;            /* completed restart cycles */
  int precond_applies;
  int status;              /* same value the solve returned */
  double rel_residual;     /* ||D (f - K x)||_2 / ||D f||_2 recomputed from x at exit, D the
                              weights of the options' residual norm */
  double rel_residual_euclid;  /* ||f - K x||_2 / ||f||_2 at exit (unweighted) */
  double time_ms;          /* wall time of the solve, host clock */
  int history_len;
  double history[KKT_HISTORY_MAX];   /* Arnoldi residual estimate / ||f|| per iteration */
} kkt_stats;

typedef struct kkt_handle kkt_handle;

/* Message of the last failure on this host thread ("" if none). */
const char* kkt_last_error(void);
/* Fixed text for a status code. */
const char* kkt_status_string(int status);
/* Fill *opt with the defaults listed in kkt_options. */
int kkt_default_options(kkt_options* opt);

/*
 * Create a solver for one KKT instance on the current CUDA device (Section 2).
 * nx, ny >= 2 grid intervals (powers of two use the fast sine transform, any other size a
 * direct O(n^2) one); Nt >= 2 time steps on (0, T]; nu > 0 conductivity; omega > 0
 * regularisation weight; n_sub time subdomains, 1 <= n_sub and Nt / n_sub >= 2 (each
 * subdomain must span two steps for the linear coarse function of Eq 14). Nt need not be a
 * multiple of n_sub: subdomain s covers steps floor((s-1)Nt/n_sub)+1 .. floor(s Nt/n_sub).
 * Returns NULL on failure (kkt_last_error() says why). Allocates the preconditioner's
 * workspace; the Krylov basis is allocated at the first kkt_solve.
 */
kkt_handle* kkt_create(int nx, int ny, int Nt, double T, double nu, double omega, int n_sub);
/* Release the handle and all device memory it holds. NULL is accepted. */
void kkt_destroy(kkt_handle* h);
/* Replace the options; takes effect at the next call. Validates every field. */
int kkt_set_options(kkt_handle* h, const kkt_options* opt);
int kkt_get_options(const kkt_handle* h, kkt_options* opt);
int kkt_get_info(const kkt_handle* h, kkt_info* info);

/*
 * f = (f_u, f_z, f) of Eq 5 for a target u_target (a block, [n][j][i], values at t_n = n dt)
 * and an initial state u0 ([j][i], N doubles; NULL means 0): f_u = h u~, f_z = 0, and f is
 * u0 in its first time slice, 0 elsewhere. Pointers may be host or device memory
 * (detected per pointer); host buffers are copied synchronously.
 */
int kkt_build_rhs(kkt_handle* h, const double* u_target, const double* u0, double* f, void* stream);

/* y = K x (Eq 5), x and y full KKT vectors (3V). Fused single pass; asynchronous. */
int kkt_matvec(kkt_handle* h, const double* x, double* y, void* stream);

/*
 * y = P^{-1} r for the block preconditioner of Eq 7: y_u = r_u / h, y_z = r_z / (omega h),
 * y_w = S-hat_2level^{-1} r_w (Eqs 13-15 with the options' coarse/variant/pou). Full KKT
 * vectors; asynchronous; uses the handle's workspace, so calls on one handle must not overlap.
 */
int kkt_precond_apply(kkt_handle* h, const double* r, double* y, void* stream);

/*
 * Solve K x = f with right-preconditioned flexible GMRES(restart) (Section 4), minimising the
 * residual in the options' norm and stopping when ||D (f - K x)|| / ||D f|| <= tol (checked on
 * the recomputed residual) or after maxit iterations. x holds the initial guess on entry and the solution on exit. f and x may be
 * host or device memory (detected per pointer; host data is staged through the handle).
 * Synchronises `stream`. Returns KKT_OK, KKT_NOT_CONVERGED (x = last iterate), or an error
 * (KKT_ERR_NONFINITE if f or an iterate is not finite, KKT_ERR_BREAKDOWN on a zero
 * Hessenberg pivot before convergence). stats may be NULL.
 */
int kkt_solve(kkt_handle* h, const double* f, double* x, double tol, int maxit,
              kkt_stats* stats, void* stream);

/* How kkt_solve moves host vectors (f in, x in and out) to and from the device. */
enum kkt_staging {
  /* pinned (page-locked) host buffers are read and written by a copy kernel through their
   * device mapping: on a coherent CPU-GPU link the SMs reach a higher rate than the copy
   * engine; pageable buffers go through cudaMemcpyAsync. The default. */
  KKT_STAGING_AUTO = 0,
  /* every host buffer through cudaMemcpyAsync (the copy engine) */
  KKT_STAGING_COPY_ENGINE = 1
};
/* Takes effect at the next kkt_solve; KKT_ERR_INVALID_ARG for another value. */
int kkt_set_staging(kkt_handle* h, int mode);

/* How the FP64 sine transforms are computed (kkt_dst2d and every FP64 preconditioner apply). */
enum kkt_dst_method {
  /* chosen at kkt_create by timing the candidates (the default): the tile height or the
   * thread-per-line transform per direction, then, on square grids of 64 to 256 intervals, the
   * tensor-core transform against those as a whole 2D transform */
  KKT_DST_AUTO = 0,
  /* tiles of lines in shared memory: the half-length FFT when the number of intervals is a
   * power of two (>= 4), on about P / 4 lanes per line (one warp per line from 256 intervals
   * up, several short lines per warp below); else the direct sum, one warp per line */
  KKT_DST_TILES = 1,
  /* one thread per line, the direct sum: lines of at most 31 points (n <= 32) */
  KKT_DST_LANE = 2,
  /* FP64-accurate dense transform on the tcgen05 tensor cores: every line and every column of
   * the DST matrix is scaled by its own power of two and cut into seven 7-bit digit planes
   * (exact in BF16); the digit-plane products accumulate exactly in FP32 and are recombined
   * in 64-bit integers (error-free splitting after Ozaki, Ogita, Oishi and Rump, 2012). Error
   * about 2^-46 of each output's line scale. Square grids with nx - 1 <= 255; holds digit
   * planes of 14 bytes and one FP64 buffer per point of a block. */
  KKT_DST_TENSOR = 3
};
/* Re-selects the method (KKT_DST_AUTO re-runs the timing). KKT_ERR_UNSUPPORTED for
 * KKT_DST_LANE when a direction has more than 31 points, and for KKT_DST_TENSOR on a
 * non-square grid or lines of more than 255 points. */
int kkt_set_dst_method(kkt_handle* h, int method);
/* The FP64 transform method in use (after KKT_DST_AUTO's timing): KKT_DST_TENSOR, KKT_DST_LANE
 * when at least one direction runs thread-per-line, else KKT_DST_TILES. */
int kkt_get_dst_method(const kkt_handle* h, int* method);

/* kkt_solve from the initial guess x_0 = 0: x is output only (its contents on entry are not
 * read, and a host x is not uploaded). Otherwise identical, including the iterates. */
int kkt_solve_zero_guess(kkt_handle* h, const double* f, double* x, double tol, int maxit,
                         kkt_stats* stats, void* stream);

/* ---- single steps of the path (device pointers, asynchronous) ------------------------- */

/* out = Q in for every time slice: the orthonormal 2D DST-I along x then y (Q^2 = I), which
 * diagonalises the 5-point Laplacian of Eq 2. Blocks: in [n][j][i], out [n][l][k] (k the x mode,
 * fastest). FP64 precision: a half-length FFT per line for power-of-two interval counts, the
 * direct sum otherwise or for short lines, or the FP64-accurate digit-plane GEMMs on the tensor
 * cores (kkt_set_dst_method; chosen at create where they time faster); in == out allowed. BF16 / TF32
 * precision (square grids): the two tensor-core GEMMs with Q, operands rounded to BF16 (the
 * intermediate too) or TF32, FP32 accumulation; in and out must not overlap. */
int kkt_dst2d(kkt_handle* h, const double* in, double* out, void* stream);

/* y = S-hat x = Jhat M_u^{-1} Jhat^T x (Eq 7), blocks. */
int kkt_schur_apply(kkt_handle* h, const double* x, double* y, void* stream);

/* y = S-hat_2level^{-1} r (Eqs 13-15, per the options), blocks: the w-block of P^{-1}. */
int kkt_schur_precond_apply(kkt_handle* h, const double* r, double* y, void* stream);

/* x0 = R_0^T S_0^{-1} R_0 r, the coarse correction alone (Eq 14 and the operator after it),
 * blocks. Needs coarse = KKT_COARSE_EXACT. */
int kkt_coarse_apply(kkt_handle* h, const double* r, double* x0, void* stream);

/* out[k] = <V_k, w> for k < count and out[count] = <w, w>, with V_k = V + k * stride; the
 * classical Gram-Schmidt multi-dot of the FGMRES Arnoldi step (Section 4). V, w and out are
 * device pointers (out: count + 1 doubles); 1 <= count <= 32, n >= 1, stride >= n. FP64,
 * deterministic (fixed grid, two-stage reduction through the handle's scratch). Asynchronous. */
int kkt_multidot(kkt_handle* h, const double* V, long long stride, int count, const double* w, long long n,
                 double* out, void* stream);

/*
 * kkt_multidot without any device allocation: the paper has no counterpart; this entry point
 * serves callers that cannot call cudaMalloc, such as a host application whose device memory
 * is owned by another allocator (a framework's caching pool, a fixed arena reserved at start-up)
 * or a loop that must not allocate. The caller passes V, w and out as for kkt_multidot (no
 * handle). The per-block partial sums live in a file-scope device array of 270,336 bytes (1024
 * blocks x 33 columns of doubles) that every GPU loading this library holds until the process
 * exits; hence count is limited to 32 and larger counts are rejected with KKT_ERR_INVALID_ARG.
 * The first call on a device looks up that array's device address (cudaGetSymbolAddress, with
 * the device current); make that first call before any stream capture. All calls share the
 * array and it keeps the last call's contents; each call writes every slot it reads before
 * reading it, so no clearing is needed, but calls that overlap on the GPU (on different
 * streams, or from different threads) race on the array and must be serialised by the caller.
 * Calls no cudaMalloc, cudaFree or allocating library routine.
 */
int kkt_multidot_noalloc(const double* V, long long stride, int count, const double* w, long long n,
                         double* out, void* stream);

/* Test hook for the reduced-precision forms' failure path, injected from the host: writes the
 * device flag that a tensor-core transform sets when one of its bounded pipeline waits runs out
 * (no kernel is made to wait). The next kkt_solve on the handle then returns KKT_ERR_TIMEOUT and
 * clears the flag. KKT_ERR_INVALID_ARG on an FP64 handle. Synchronous. */
int kkt_inject_tc_timeout(kkt_handle* h);

/* ---- learned coarse correction (not in the paper) ---------------------------------------
 * A two-hidden-layer ReLU network maps a low sine mode's coarse right-hand side c = R_0 r
 * (Eq 14; normalised, 2 n_sub values) and the mode's features (log dt nu lambda,
 * log dt/sqrt(omega)) to a direction d of its coarse correction S_0^{-1} R_0 r. An exact
 * one-dimensional minimal-residual step with the mode's coarse operator G = h S_0(mu) sets the
 * magnitude, alpha = (G d)^T c / ||G d||^2, so the correction alpha d never increases the coarse
 * residual; a residual guard (||c - alpha G d|| <= ||c|| / 2) falls back to the exact coarse
 * solve. Trained on the GPU on coarse solves generated by the method (restriction of seeded
 * residual time series, exact block-Thomas solve) with Adam, first on the squared error to the
 * unit target, then on the guard's quantity ||c - alpha G d||^2 / ||c||^2. Weights BF16 for
 * inference, FP32 accumulation; FP32 master weights for training. */
typedef struct kkt_mlp kkt_mlp;

typedef struct kkt_mlp_config {
  int nx;        /* grid intervals of the training geometry (its sine spectrum gives lambda) */
  int Nt;        /* time steps */
  int n_sub;     /* subdomains; network input 2 n_sub + 2, output 2 n_sub */
  int modes;     /* learned modes per direction: k, l < modes */
  int width;     /* hidden width */
  int seed;      /* initialisation and sampling seed */
  int samples;   /* training samples (rounded up to whole (nu, omega) draws of modes^2) */
  int epochs;    /* epochs on the squared error to the unit target */
  int batch;
  double T;
  double nu_lo, nu_hi;        /* nu log-uniform on [nu_lo, nu_hi] */
  double omega_lo, omega_hi;  /* omega log-uniform on [omega_lo, omega_hi] */
  double lr;                  /* Adam step (x 0.3 for the last third of each phase's epochs) */
  int resid_epochs;           /* then epochs on the coarse residual after the minimal-residual step */
} kkt_mlp_config;

typedef struct kkt_mlp_train_stats {
  int samples, steps;
  double final_train_loss, val_loss, val_cosine;   /* val: held-out tenth, BF16 weights */
  double val_resid;          /* mean of ||c - alpha G d||^2 / ||c||^2 on the held-out samples */
  double val_within_guard;   /* fraction of them the guard keeps (that ratio <= 1/4) */
} kkt_mlp_train_stats;

int kkt_mlp_default_config(kkt_mlp_config* cfg);
kkt_mlp* kkt_mlp_create(const kkt_mlp_config* cfg);   /* NULL on failure */
void kkt_mlp_destroy(kkt_mlp* m);
/* Parameters as one FP32 array: W1 [width][2 n_sub + 2], b1, W2 [width][width], b2,
 * W3 [2 n_sub][width], b3 (host memory). */
int kkt_mlp_param_count(const kkt_mlp* m, long long* count);
int kkt_mlp_get_config(const kkt_mlp* m, kkt_mlp_config* cfg);
int kkt_mlp_set_params(kkt_mlp* m, const float* host, long long count);
int kkt_mlp_get_params(const kkt_mlp* m, float* host, long long count);
/* Y = net(X) for a batch (device FP32, rows of 2 n_sub + 2 / 2 n_sub); use_bf16 selects the
 * BF16 weights. */
int kkt_mlp_forward(kkt_mlp* m, const float* X, float* Y, int batch, int use_bf16, void* stream);
/* loss = 1/(2 batch) sum ||net(X) - T||^2 (FP32 weights); grad (device, parameter layout) may be
 * NULL; *loss is written after synchronising `stream` when loss != NULL. */
int kkt_mlp_loss_grad(kkt_mlp* m, const float* X, const float* T, int batch, float* grad, double* loss,
                      void* stream);
/* The coarse-residual loss: loss = 1/batch sum_b ||c_b - alpha_b G(mu_b) d_b||^2 / ||c_b||^2 with
 * d_b = net(X_b) (FP32 weights), c_b the first 2 n_sub entries of X_b, alpha_b the
 * minimal-residual step and G(mu) the coarse operator of a mode with Jhat diagonal mu on the
 * network's training decomposition (config Nt, n_sub; balanced split, left partition of unity).
 * mu: device FP64 [batch]. grad and loss as for kkt_mlp_loss_grad. */
int kkt_mlp_resid_loss_grad(kkt_mlp* m, const float* X, const double* mu, int batch, float* grad, double* loss,
                            void* stream);
/* The training pairs the method generates, for checking: per sample b of `count`, the mode's time
 * series r[n * count + b] (n = 0..Nt-1, device FP64) is restricted, c_b = R_0 r_b [2 n_sub]
 * (Eq 14), and x_b = G(mu_b)^{-1} c_b by the block-Thomas elimination of the coarse system.
 * c, x: device FP64 [count][2 n_sub]. Allocates a scratch of 40 n_sub bytes per sample and
 * synchronises `stream`. */
int kkt_mlp_coarse_data(kkt_mlp* m, const double* r, const double* mu, long long count, double* c, double* x,
                        void* stream);
/* One Adam step (beta 0.9, 0.999, eps 1e-8) on the batch. */
int kkt_mlp_adam_step(kkt_mlp* m, const float* X, const float* T, int batch, double lr, double* loss,
                      void* stream);
/* Generate the training set on the GPU and train (synchronises). */
int kkt_mlp_train(kkt_mlp* m, kkt_mlp_train_stats* stats, void* stream);
int kkt_mlp_save(const kkt_mlp* m, const char* path);
kkt_mlp* kkt_mlp_load(const char* path);
/* Use the network for coarse = KKT_COARSE_LEARNED on this handle (the handle does not own it;
 * keep it alive). mode 0: the network's corrections with the guard (exact solve where the guard
 * rejects); mode 1: no coarse correction on the learned modes (the ablation); mode 2: the
 * network's corrections always, no guard and no exact fallback (what the network alone gives).
 * Needs 2 n_sub of the handle = the network's output and modes <= min(nx, ny) - 1. */
int kkt_attach_mlp(kkt_handle* h, kkt_mlp* m, int mode);
/* Learned-mode coarse corrections since the last call: kept (applied) and, in mode 0, replaced
 * by the exact solve; in mode 2 `fallback` counts the applied corrections the guard would have
 * rejected. */
int kkt_learned_stats(kkt_handle* h, long long* kept, long long* fallback, int reset);

/* ---- batched form: many independent instances of uneven sizes ------------------------
 *
 * Not part of the paper's method: a throughput form that solves many independent KKT systems
 * (Eq 5) with the same preconditioner and FGMRES as kkt_solve. Instances are packed into waves
 * that fit in device memory; inside a wave every Arnoldi step runs each phase (sine transforms,
 * coarse solve, sweeps, matvec, Gram-Schmidt) as ONE launch over all instances of the wave, and
 * the preconditioner + matvec phase of each step index is captured once as a CUDA graph and
 * replayed. FP64 only, exact or one-level coarse level; instances keep their own sizes and
 * parameters. Iterations and residual histories equal those of kkt_solve up to rounding.
 */
#define KKT_BATCH_MAX 256
typedef struct kkt_instance {
  int nx, ny, Nt, n_sub;
  double T, nu, omega;
} kkt_instance;

typedef struct kkt_batch_stats {
  int solo;                /* instances at or above the single-solve threshold, solved one by one */
  int waves;               /* memory waves the other instances were packed into */
  int graphs;              /* CUDA graphs captured (one per wave and Arnoldi step index used) */
  long long graph_launches;
  int tile_lines;          /* sine-transform tile height the autotuner chose */
  int sweep_block;         /* sweep block size the autotuner chose */
  double tune_ms_dst[3];   /* autotuner timings of tile heights 8, 16, 32 (ms per forward pair) */
  double tune_ms_sweep[3]; /* and of sweep blocks 64, 128, 256 */
  double time_ms;          /* wall time, host clock */
  int iterations[KKT_BATCH_MAX];
  int status[KKT_BATCH_MAX];
  double rel_residual[KKT_BATCH_MAX];  /* recomputed from x at exit, options' residual norm */
} kkt_batch_stats;

typedef struct kkt_batch kkt_batch;

/* count (1..KKT_BATCH_MAX) instances with the shared options (NULL = defaults; precision must
 * be FP64 and coarse EXACT or NONE, else NULL with KKT_ERR_UNSUPPORTED). NULL on failure. */
kkt_batch* kkt_batch_create(int count, const kkt_instance* inst, const kkt_options* opt);
void kkt_batch_destroy(kkt_batch* b);
int kkt_batch_get_info(const kkt_batch* b, int i, kkt_info* info);
/* Cap the Krylov storage of one wave at `bytes` (0: 85% of the free device memory at solve time,
 * the default). A smaller cap gives more, smaller waves; an instance larger than the cap fails
 * the solve with KKT_ERR_OOM. */
int kkt_batch_set_memory_limit(kkt_batch* b, long long bytes);
/* on != 0 (default): the preconditioner + matvec phase of each Arnoldi step index is captured
 * once per wave as a CUDA graph and replayed; 0: its kernels are launched directly every step
 * (same kernels and results; their device time is then profiled per kernel class). */
int kkt_batch_set_graphs(kkt_batch* b, int on);
/* Instances with at least `points` unknowns per block (V) fill the GPU on their own: they are
 * solved one after another with kkt_solve's path (their Krylov storage released after each),
 * before the batched waves of the others. Default 2^20 (measured: batching gains 2.6x below
 * about 5e5 unknowns per block and loses above about 1e6); 0 batches every instance. */
int kkt_batch_set_single_threshold(kkt_batch* b, long long points);
/* The FP64 transform method of every instance, as kkt_set_dst_method sets it for one handle
 * (default: each instance's own create-time timing). In the batched waves, an instance whose
 * transforms run on the tensor cores and whose GEMM passes have at least one tile per SM is
 * transformed alone (one kkt_dst2d each, inside the step's graph); the others share the line-tile
 * launches. Returns the first instance's error (KKT_ERR_UNSUPPORTED for KKT_DST_TENSOR on an
 * instance it does not apply to); instances before it keep the new method. */
int kkt_batch_set_dst_method(kkt_batch* b, int method);
/* Solve K_i x_i = f_i for every instance. f, x: host arrays of count DEVICE pointers, 3 V_i
 * doubles each; x_i holds the initial guess on entry. Synchronises `stream`. Returns KKT_OK
 * when every instance converged, KKT_NOT_CONVERGED if some stopped at maxit, else the most
 * severe per-instance error; per-instance outcomes are in stats. Device memory for the Krylov
 * bases is taken per wave (about 8 (4 restart + 3) V_i bytes per instance) and released. */
int kkt_batch_solve(kkt_batch* b, const double* const* f, double* const* x, double tol, int maxit,
                    kkt_batch_stats* stats, void* stream);

/* ---- instrumentation ------------------------------------------------------------------ */

/* Kernel classes counted and timed by the library (process-wide, all handles). */
enum kkt_kernel_class {
  KKT_K_DST = 0,       /* 2D sine transform passes (rows or columns) */
  KKT_K_COARSE = 1,    /* coarse restriction + block-tridiagonal coarse solve */
  KKT_K_SWEEP = 2,     /* per-subdomain forward/backward sweeps (+ coarse prolongation) */
  KKT_K_MATVEC = 3,    /* KKT matvec and other stencil passes */
  KKT_K_MULTIDOT = 4,  /* Gram-Schmidt multi-dot */
  KKT_K_UPDATE = 5,    /* Gram-Schmidt update + norm */
  KKT_K_AXPY = 6,      /* solution update and elementwise passes */
  KKT_K_REDUCE = 7,    /* reduction finalisation and norms */
  KKT_K_GRAPH = 8,     /* a replayed CUDA graph (batched form): its kernels are counted in their
                          own classes, its time, flops and bytes here */
  KKT_K_PACK = 9,      /* reduced-precision forms: FP64 input split into tensor-core operands */
  KKT_K_COUNT = 10
};

typedef struct kkt_kernel_stats {
  long long launches[KKT_K_COUNT];  /* kernels launched, always counted */
  double ms[KKT_K_COUNT];           /* summed device time (CUDA events), only while timing is on */
  long long timed[KKT_K_COUNT];     /* launches that were timed */
  double flops[KKT_K_COUNT];        /* algorithmic floating-point operations of the timed launches */
  double bytes[KKT_K_COUNT];        /* algorithmic device-memory bytes of the timed launches */
} kkt_kernel_stats;

/* Turn per-launch CUDA-event timing on (1) or off (0); each timed launch records two events on
 * its stream. Process-wide; not thread-safe against concurrent solves. */
int kkt_profile_enable(int on);
/* Copy the counters (synchronising on the pending timing events) and, if reset != 0, zero them. */
int kkt_profile_read(kkt_kernel_stats* out, int reset);

/* Peak-rate probe (no counterpart in the paper; the denominator of the FP64 and FP32 rooflines):
 * a bounded loop of independent fused multiply-adds on 8 CTAs of 256 threads per SM, about 20 ms
 * per launch, best of 5 timed launches with CUDA events on `stream` after one warm-up.
 * precision 0: FP64, 1: FP32; *flops_per_s = 2 x FMAs / s. Synchronises `stream`; allocates and
 * frees a small sink buffer. */
int kkt_probe_fma_rate(int precision, double* flops_per_s, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* KKT_H */
