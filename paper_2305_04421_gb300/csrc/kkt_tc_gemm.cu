// Sine transforms as dense GEMMs on the 5th-generation tensor cores (tcgen05), for the
// reduced-precision forms of the preconditioner: every implicit spatial step of the sweeps
// of Eq 13 is diagonalised by the 2D DST-I, here applied as products with the DST matrix Q.
//
// One kernel serves all four transforms of a preconditioner apply. Input A is a stack of S
// slices, each P x P (rows x K, K contiguous), B is Q (P x P, symmetric, zero-padded past
// n-1), and the output is stored TRANSPOSED per slice:
//     O[s][c][r] = sum_k A[s][r][k] Q[k][c]
// so the next transform again contracts along the contiguous axis, and the stores of the
// epilogue are coalesced (32 consecutive r per warp).
//
// Split operands (forward transforms): A = A_hi + A_lo and Q = Q_hi + Q_lo, each part in the
// operand type, and the tile accumulates A_hi Q_hi + A_hi Q_lo + A_lo Q_hi in the same TMEM
// accumulator (the lo x lo term, about 2^-16 (BF16) or 2^-22 (TF32) of the product, is
// dropped). The forward transform's rounding error is spread evenly over all modes and the
// sweeps then amplify the low modes by up to (mu_max / mu_min)^2, so the forward transforms
// need this extra accuracy; the inverse transforms do not (their error is relative to their
// own output) and use single operands.
//
// The transforms run the persistent, warp-specialised kernel: one CTA per SM walks its tiles
// (128 x TILE_N outputs each); warp 0 lane 0 streams A and B chunks of 128 bytes of K through
// a shared-memory ring with TMA (128B swizzle) and mbarriers, warp 1 lane 0 issues tcgen05.mma
// (M = 128, N = TILE_N, K = 16 for BF16 / 8 for TF32, FP32 accumulation) into one of two TMEM
// accumulators, and warps 2-5 read the other accumulator back with tcgen05.ld (each warp its
// 32-lane quarter) and store, so the epilogue of one tile overlaps the loads and MMAs of the
// next. The one-tile-per-CTA kernel below it is the same pipeline without that overlap.
// Every mbarrier wait is bounded (about 2 s of clock); on a timeout the kernel records an
// error flag, skips its remaining work, still waits (bounded) for its own copies and MMAs,
// frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "kkt_internal.cuh"

namespace kkt {
namespace {

constexpr int kTileM = 128;
constexpr int kStages = 2;
constexpr int kChunkBytes = 128;                      // K bytes per TMA box row (one swizzle span)
constexpr long long kWaitCycles = 4000000000LL;       // ~2 s at 2 GHz
// the transforms run the persistent, warp-specialised kernel (false: one tile per CTA)
constexpr bool kPersistentGemm = true;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: true on success, false after ~2 s.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128B swizzle, 8-row atoms 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
  const uint64_t addr = smem_u32(p);
  uint64_t d = (addr & 0x3FFFFull) >> 4;       // start address, bits [0,14)
  d |= 1ull << 16;                             // leading byte offset (unused for swizzled K-major)
  d |= (1024ull >> 4) << 32;                   // stride byte offset: 8 rows x 128 B
  d |= 1ull << 46;                             // descriptor version
  d |= 2ull << 61;                             // swizzle: 128B
  return d;
}

// The same descriptor for 64-byte K rows with 64B swizzle: 8-row atoms 512 B apart.
__device__ __forceinline__ uint64_t smem_desc64(const void* p) {
  const uint64_t addr = smem_u32(p);
  uint64_t d = (addr & 0x3FFFFull) >> 4;       // start address, bits [0,14)
  d |= 1ull << 16;                             // leading byte offset (unused for swizzled K-major)
  d |= (512ull >> 4) << 32;                    // stride byte offset: 8 rows x 64 B
  d |= 1ull << 46;                             // descriptor version
  d |= 4ull << 61;                             // swizzle: 64B
  return d;
}

template <typename TIn>
struct MmaKind;

template <>
struct MmaKind<__nv_bfloat16> {
  static constexpr int kFormat = 1;            // BF16
  static constexpr int kUmmaK = 16;            // 32 bytes of K per instruction
  static __device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
};

template <>
struct MmaKind<float> {
  static constexpr int kFormat = 2;            // TF32
  static constexpr int kUmmaK = 8;
  static __device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
};

// Instruction descriptor: FP32 accumulator, A and B of the given format, both K-major.
template <typename TIn, int N>
__host__ __device__ constexpr uint32_t instr_desc() {
  return (1u << 4)                                              // D format: F32
         | (static_cast<uint32_t>(MmaKind<TIn>::kFormat) << 7)   // A format
         | (static_cast<uint32_t>(MmaKind<TIn>::kFormat) << 10)  // B format
         | (static_cast<uint32_t>(N >> 3) << 17)                 // N / 8
         | (static_cast<uint32_t>(kTileM >> 4) << 24);           // M / 16
}

struct TcParams {
  int P;              // padded transform size (multiple of 128)
  int slices;
  int valid;          // output mode 2: rows/cols < valid are stored, into a valid x valid slice
  void* out;
  void* out_lo;       // output mode 3: the lo part
  int* err;           // device error flag (set to 1 on a wait timeout)
};

enum OutMode { kOutBF16 = 0, kOutF32 = 1, kOutF64 = 2, kOutSplit = 3 };

// TF32 rounding of an FP32 value (10 explicit mantissa bits, ties away from zero)
__device__ __forceinline__ float tf32_round(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// FP64 -> FP32 conversion in integer arithmetic on the two 32-bit halves of the bit pattern. On
// this part the FP64 pipe (2 instructions per clock per SM) also executes F2F conversions, and a
// version on 64-bit integers still kept that pipe 78 % busy under ncu, so the rounding uses
// 32-bit operations only: the top 23 fraction bits come from the high word and the top 3 bits of
// the low word, the other 29 bits of the low word decide the rounding (to nearest, ties to
// even). Values below FP32's normal range are flushed to zero, values above it become
// infinities, NaNs stay NaNs.
__device__ __forceinline__ float f64_to_f32_rne(double d) {
  const unsigned hi = static_cast<unsigned>(__double2hiint(d)), lo = static_cast<unsigned>(__double2loint(d));
  const unsigned sign = hi & 0x80000000u;
  const int e = static_cast<int>((hi >> 20) & 0x7ffu);
  unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const unsigned rest = lo & 0x1FFFFFFFu;
  if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | ((m | rest) ? 0x00400000u : 0u));
  int e32 = e - 1023 + 127;
  if (e32 <= 0) return __uint_as_float(sign);
  m += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
  if (m >> 23) {
    m = 0;
    ++e32;
  }
  if (e32 >= 255) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | (static_cast<unsigned>(e32) << 23) | m);
}

// hi + lo split of a value in the operand type
template <typename TIn>
struct Split;
template <>
struct Split<__nv_bfloat16> {
  static __device__ __forceinline__ void make(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
};
template <>
struct Split<float> {
  static __device__ __forceinline__ void make(float v, float& hi, float& lo) {
    hi = tf32_round(v);
    lo = v - hi;
  }
};

template <typename TIn, int TILE_N, int OUT, bool SPLIT>
__global__ void __launch_bounds__(128, 1)
    tc_dst_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                       const __grid_constant__ CUtensorMap tmAlo, const __grid_constant__ CUtensorMap tmBlo,
                       TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int A_BYTES = kTileM * kChunkBytes;
  constexpr int B_BYTES = TILE_N * kChunkBytes;
  constexpr int PART = A_BYTES + B_BYTES;                 // one hi (or lo) pair of tiles
  constexpr int STAGE = SPLIT ? 2 * PART : PART;
  constexpr int KCHUNK = kChunkBytes / static_cast<int>(sizeof(TIn));   // elements of K per chunk
  constexpr int UMMA_K = MmaKind<TIn>::kUmmaK;
  constexpr int K_STEPS = KCHUNK / UMMA_K;                               // 4 MMAs per chunk
  constexpr uint32_t IDESC = instr_desc<TIn, TILE_N>();
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * STAGE);
  uint64_t* empty = full + kStages;
  uint64_t* done = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntile_c = p.P / TILE_N, ntile_r = p.P / kTileM;
  const int tile = blockIdx.x;
  const int s = tile / (ntile_c * ntile_r);
  const int rem = tile - s * ntile_c * ntile_r;
  const int rt = rem / ntile_c, ct = rem - rt * ntile_c;
  const int nchunks = p.P / KCHUNK;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TILE_N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  int issued = 0;       // chunks whose TMA copies were issued (producer thread)
  if (warp == 0 && lane == 0) {
    for (int c = 0; c < nchunks; ++c) {
      const int st = c % kStages;
      if (c >= kStages && !mbar_wait(empty + st, ((c / kStages) & 1) ^ 1)) {
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      uint8_t* sa = smem + st * STAGE;
      mbar_expect_tx(full + st, STAGE);
      tma_load_2d(sa, &tmA, c * KCHUNK, s * p.P + rt * kTileM, full + st);
      tma_load_2d(sa + A_BYTES, &tmB, c * KCHUNK, ct * TILE_N, full + st);
      if (SPLIT) {
        tma_load_2d(sa + PART, &tmAlo, c * KCHUNK, s * p.P + rt * kTileM, full + st);
        tma_load_2d(sa + PART + A_BYTES, &tmBlo, c * KCHUNK, ct * TILE_N, full + st);
      }
      ++issued;
    }
  } else if (warp == 1 && lane == 0) {
    for (int c = 0; c < nchunks; ++c) {
      const int st = c % kStages;
      if (!mbar_wait(full + st, (c / kStages) & 1)) {
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint8_t* sa = smem + st * STAGE;
      const uint64_t da = smem_desc(sa), db = smem_desc(sa + A_BYTES);
#pragma unroll
      for (int kk = 0; kk < K_STEPS; ++kk) {
        // advance 32 bytes of K inside the 128-byte swizzle row: +2 in the encoded address
        MmaKind<TIn>::mma(tmem, da + 2ull * kk, db + 2ull * kk, IDESC, (c | kk) != 0);
      }
      if (SPLIT) {
        const uint64_t dal = smem_desc(sa + PART), dbl = smem_desc(sa + PART + A_BYTES);
#pragma unroll
        for (int kk = 0; kk < K_STEPS; ++kk) {
          MmaKind<TIn>::mma(tmem, da + 2ull * kk, dbl + 2ull * kk, IDESC, 1u);    // A_hi Q_lo
          MmaKind<TIn>::mma(tmem, dal + 2ull * kk, db + 2ull * kk, IDESC, 1u);    // A_lo Q_hi
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   ::"r"(smem_u32(empty + st)) : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(done)) : "memory");
  }
  __syncwarp();
  // every thread: wait for the last MMA (the commit on `done` arrives after all issued MMAs)
  const bool ok = mbar_wait(done, 0);
  if (!ok) *abort_flag = 1;
  __syncthreads();
  if (*abort_flag) {
    if (threadIdx.x == 0) atomicExch(p.err, 1);
    // let the copies this CTA issued land before its shared memory is released
    // (only the last kStages issued chunks can still be in flight: an older stage was refilled
    // only after its MMAs, and so its copy, had completed)
    if (warp == 0 && lane == 0) {
      for (int c = issued > kStages ? issued - kStages : 0; c < issued; ++c)
        mbar_wait(full + (c % kStages), (c / kStages) & 1);
    }
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int r = rt * kTileM + warp * 32 + lane;
    const uint32_t tbase = tmem + (static_cast<uint32_t>(warp * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < TILE_N; c0 += 16) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tbase + c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const int c = ct * TILE_N + c0 + t;
        const float val = __uint_as_float(v[t]);
        if (OUT == kOutBF16) {
          reinterpret_cast<__nv_bfloat16*>(p.out)[(static_cast<long long>(s) * p.P + c) * p.P + r] = __float2bfloat16_rn(val);
        } else if (OUT == kOutSplit) {
          TIn hi, lo;
          Split<TIn>::make(val, hi, lo);
          const long long o = (static_cast<long long>(s) * p.P + c) * p.P + r;
          reinterpret_cast<TIn*>(p.out)[o] = hi;
          reinterpret_cast<TIn*>(p.out_lo)[o] = lo;
        } else if (OUT == kOutF32) {
          reinterpret_cast<float*>(p.out)[(static_cast<long long>(s) * p.P + c) * p.P + r] = val;
        } else {
          if (c < p.valid && r < p.valid)
            reinterpret_cast<double*>(p.out)[(static_cast<long long>(s) * p.valid + c) * p.valid + r] = static_cast<double>(val);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TILE_N));
}

// Epilogue store of one accumulator value (row r, column c of slice s) in the output mode.
template <typename TIn, int OUT>
__device__ __forceinline__ void store_out(const TcParams& p, int s, int r, int c, float val) {
  if (OUT == kOutBF16) {
    reinterpret_cast<__nv_bfloat16*>(p.out)[(static_cast<long long>(s) * p.P + c) * p.P + r] = __float2bfloat16_rn(val);
  } else if (OUT == kOutSplit) {
    TIn hi, lo;
    Split<TIn>::make(val, hi, lo);
    const long long o = (static_cast<long long>(s) * p.P + c) * p.P + r;
    reinterpret_cast<TIn*>(p.out)[o] = hi;
    reinterpret_cast<TIn*>(p.out_lo)[o] = lo;
  } else if (OUT == kOutF32) {
    reinterpret_cast<float*>(p.out)[(static_cast<long long>(s) * p.P + c) * p.P + r] = val;
  } else {
    if (c < p.valid && r < p.valid)
      reinterpret_cast<double*>(p.out)[(static_cast<long long>(s) * p.valid + c) * p.valid + r] = static_cast<double>(val);
  }
}

// Persistent, warp-specialised form of the same transform: one CTA per SM walks tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...; warp 0 lane 0 streams A and Q chunks through the
// shared-memory ring (TMA), warp 1 lane 0 issues the MMAs into one of two TMEM accumulators
// (2 x TILE_N columns), and warps 2-5 read the other accumulator back and store it, so a tile's
// epilogue overlaps the next tile's loads and MMAs. Barriers: full/empty per ring stage,
// tmem_full/tmem_empty per accumulator (the four epilogue warps arrive on tmem_empty), done at
// teardown. Every wait is bounded; a timeout sets the error flag and every role stops at its
// next check; teardown waits (bounded) for the CTA's own copies and MMAs and frees TMEM.
constexpr int kPersistThreads = 192;

template <typename TIn, int TILE_N, int OUT, bool SPLIT>
__global__ void __launch_bounds__(kPersistThreads, 1)
    tc_dst_gemm_persistent(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                           const __grid_constant__ CUtensorMap tmAlo, const __grid_constant__ CUtensorMap tmBlo,
                           TcParams p, int stages) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int A_BYTES = kTileM * kChunkBytes;
  constexpr int B_BYTES = TILE_N * kChunkBytes;
  constexpr int PART = A_BYTES + B_BYTES;
  constexpr int STAGE = SPLIT ? 2 * PART : PART;
  constexpr int KCHUNK = kChunkBytes / static_cast<int>(sizeof(TIn));
  constexpr int UMMA_K = MmaKind<TIn>::kUmmaK;
  constexpr int K_STEPS = KCHUNK / UMMA_K;
  constexpr uint32_t IDESC = instr_desc<TIn, TILE_N>();
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + stages * STAGE);
  uint64_t* empty = full + stages;
  uint64_t* tfull = empty + stages;        // [2]
  uint64_t* tempty = tfull + 2;            // [2]
  uint64_t* done = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntile_c = p.P / TILE_N, ntile_r = p.P / kTileM;
  const int per_slice = ntile_c * ntile_r;
  const long long ntiles = static_cast<long long>(p.slices) * per_slice;
  const int nchunks = p.P / KCHUNK;

  if (threadIdx.x == 0) {
    for (int i = 0; i < stages; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(tfull + i, 1);
      mbar_init(tempty + i, 4);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * TILE_N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  long long issued = 0;   // chunks whose copies were issued (producer)
  if (warp == 0) {
    if (lane == 0) {
      long long g = 0;
      for (long long tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x) {
        const int s = static_cast<int>(tile / per_slice);
        const int rem = static_cast<int>(tile - static_cast<long long>(s) * per_slice);
        const int rt = rem / ntile_c, ct = rem - rt * ntile_c;
        for (int c = 0; c < nchunks; ++c, ++g) {
          const int st = static_cast<int>(g % stages);
          if (g >= stages && !mbar_wait(empty + st, static_cast<uint32_t>(((g / stages) & 1) ^ 1))) {
            *abort_flag = 1;
            break;
          }
          if (*abort_flag) break;
          uint8_t* sa = smem + st * STAGE;
          mbar_expect_tx(full + st, STAGE);
          tma_load_2d(sa, &tmA, c * KCHUNK, s * p.P + rt * kTileM, full + st);
          tma_load_2d(sa + A_BYTES, &tmB, c * KCHUNK, ct * TILE_N, full + st);
          if (SPLIT) {
            tma_load_2d(sa + PART, &tmAlo, c * KCHUNK, s * p.P + rt * kTileM, full + st);
            tma_load_2d(sa + PART + A_BYTES, &tmBlo, c * KCHUNK, ct * TILE_N, full + st);
          }
          ++issued;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      long long g = 0;
      int local = 0;
      for (long long tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x, ++local) {
        const int acc = local & 1;
        if (local >= 2 && !mbar_wait(tempty + acc, static_cast<uint32_t>(((local >> 1) & 1) ^ 1))) {
          *abort_flag = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t tacc = tmem + static_cast<uint32_t>(acc * TILE_N);
        for (int c = 0; c < nchunks; ++c, ++g) {
          const int st = static_cast<int>(g % stages);
          if (!mbar_wait(full + st, static_cast<uint32_t>((g / stages) & 1))) {
            *abort_flag = 1;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint8_t* sa = smem + st * STAGE;
          const uint64_t da = smem_desc(sa), db = smem_desc(sa + A_BYTES);
#pragma unroll
          for (int kk = 0; kk < K_STEPS; ++kk)
            MmaKind<TIn>::mma(tacc, da + 2ull * kk, db + 2ull * kk, IDESC, (c | kk) != 0);
          if (SPLIT) {
            const uint64_t dal = smem_desc(sa + PART), dbl = smem_desc(sa + PART + A_BYTES);
#pragma unroll
            for (int kk = 0; kk < K_STEPS; ++kk) {
              MmaKind<TIn>::mma(tacc, da + 2ull * kk, dbl + 2ull * kk, IDESC, 1u);
              MmaKind<TIn>::mma(tacc, dal + 2ull * kk, db + 2ull * kk, IDESC, 1u);
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                       ::"r"(smem_u32(empty + st)) : "memory");
        }
        if (*abort_flag) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(smem_u32(tfull + acc)) : "memory");
      }
      // completes after every MMA this thread issued
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   ::"r"(smem_u32(done)) : "memory");
    }
  } else {
    // epilogue warps 2..5: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows of the tile)
    const int quad = warp & 3;
    int local = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++local) {
      if (*abort_flag) break;
      const int acc = local & 1;
      if (!mbar_wait(tfull + acc, static_cast<uint32_t>((local >> 1) & 1))) {
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int s = static_cast<int>(tile / per_slice);
      const int rem = static_cast<int>(tile - static_cast<long long>(s) * per_slice);
      const int rt = rem / ntile_c, ct = rem - rt * ntile_c;
      const int r = rt * kTileM + quad * 32 + lane;
      const uint32_t tbase = tmem + (static_cast<uint32_t>(quad * 32) << 16) + static_cast<uint32_t>(acc * TILE_N);
#pragma unroll 1
      for (int c0 = 0; c0 < TILE_N; c0 += 16) {
        uint32_t v[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(tbase + c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int t = 0; t < 16; ++t) store_out<TIn, OUT>(p, s, r, ct * TILE_N + c0 + t, __uint_as_float(v[t]));
      }
      // this warp's reads of the accumulator are complete: release it to the MMA warp
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(tempty + acc)) : "memory");
    }
  }
  __syncwarp();
  // teardown: every MMA issued (the done commit), then, after a timeout, the producer's copies
  if (!mbar_wait(done, 0)) *abort_flag = 1;
  __syncthreads();
  if (*abort_flag) {
    if (threadIdx.x == 0) atomicExch(p.err, 1);
    if (warp == 0 && lane == 0) {
      for (long long c = issued > stages ? issued - stages : 0; c < issued; ++c)
        mbar_wait(full + static_cast<int>(c % stages), static_cast<uint32_t>((c / stages) & 1));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TILE_N));
}

// out + out_lo (P x P per slice, zero padded) = in[s][j][i] (valid x valid), split into hi and
// lo parts of the operand type (callers fold any scale downstream). No FP64 instruction: the
// value is rounded to FP32 by integer operations on its bit pattern (f64_to_f32_rne) and split
// on the FP32 pipe (Split::make: hi = v rounded to the operand's significand, lo = v - hi, exact
// in FP32). The FP32 rounding (2^-24 relative) is far below the split's own 2^-16 (BF16) and
// 2^-22 (TF32). Each thread packs two neighbouring elements of a row (one 4- or 8-byte store per
// part; P is even). Grid (P / 512 rounded up, P, slices): no 64-bit index divisions (the
// compiler builds those from FP64 arithmetic, the scarce pipe here).
template <typename TIn>
struct Pair;
template <>
struct Pair<__nv_bfloat16> {
  using T = __nv_bfloat162;
  static __device__ __forceinline__ T make(__nv_bfloat16 a, __nv_bfloat16 b) { return __halves2bfloat162(a, b); }
};
template <>
struct Pair<float> {
  using T = float2;
  static __device__ __forceinline__ T make(float a, float b) { return make_float2(a, b); }
};

template <typename TIn>
__global__ void pack_kernel(const double* __restrict__ in, TIn* __restrict__ out, TIn* __restrict__ out_lo, int P,
                            int valid) {
  const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int j = blockIdx.y;
  const long long s = blockIdx.z;
  if (i >= P) return;
  const long long t = (s * P + j) * P + i;
  float v0 = 0.f, v1 = 0.f;
  if (j < valid) {
    const double* row = in + (s * valid + j) * valid;
    const double d0 = i < valid ? row[i] : 0.0, d1 = i + 1 < valid ? row[i + 1] : 0.0;
    v0 = f64_to_f32_rne(d0);
    v1 = f64_to_f32_rne(d1);
  }
  TIn h0, l0, h1, l1;
  Split<TIn>::make(v0, h0, l0);
  Split<TIn>::make(v1, h1, l1);
  *reinterpret_cast<typename Pair<TIn>::T*>(out + t) = Pair<TIn>::make(h0, h1);
  *reinterpret_cast<typename Pair<TIn>::T*>(out_lo + t) = Pair<TIn>::make(l0, l1);
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int get_encode(EncodeFn* fn) {
  static EncodeFn cached = nullptr;
  if (!cached) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    KKT_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q));
    if (!f || q != cudaDriverEntryPointSuccess) return set_error(KKT_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    cached = reinterpret_cast<EncodeFn>(f);
  }
  *fn = cached;
  return KKT_OK;
}

// 2D tensor map over rows x P (K contiguous), box = (chunk_bytes of K) x box_rows, swizzled over
// the box's rows: 128B swizzle for 128-byte chunks, 64B swizzle for 64-byte chunks.
int make_map(CUtensorMap* map, const void* base, int elem_bytes, long long rows, int P, int box_rows,
             int chunk_bytes = kChunkBytes) {
  EncodeFn enc = nullptr;
  KKT_TRY(get_encode(&enc));
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(P), static_cast<cuuint64_t>(rows)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(P) * elem_bytes};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(chunk_bytes / elem_bytes), static_cast<cuuint32_t>(box_rows)};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                         const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         chunk_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(KKT_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string(static_cast<int>(r)));
  return KKT_OK;
}

template <typename TIn, int TILE_N, int OUT, bool SPLIT>
int launch_gemm(const CUtensorMap& a, const CUtensorMap& b, const CUtensorMap& alo, const CUtensorMap& blo,
                const TcParams& p, cudaStream_t st) {
  constexpr int PART = (kTileM + TILE_N) * kChunkBytes;
  constexpr int STAGE = SPLIT ? 2 * PART : PART;
  const long long tiles = static_cast<long long>(p.slices) * (p.P / kTileM) * (p.P / TILE_N);
  // dense GEMM with Q per slice: 2 P^3 flops (x3 for split operands); operands in, result out
  const double planes = static_cast<double>(p.slices) * p.P * p.P;
  const double out_b = OUT == kOutBF16 ? 2.0 * planes
                       : (OUT == kOutSplit ? 2.0 * sizeof(TIn) * planes
                                           : (OUT == kOutF32 ? 4.0 * planes : 8.0 * static_cast<double>(p.slices) * p.valid * p.valid));
  ProfScope ps(KKT_K_DST, st, (SPLIT ? 6.0 : 2.0) * planes * p.P, planes * sizeof(TIn) * (SPLIT ? 2 : 1) + out_b);
  if (kPersistentGemm) {
    // as many ring stages as fit beside the barriers (2 with split 256-wide tiles, up to 4)
    const int stages = std::max(2, std::min(4, static_cast<int>((220 * 1024 - 1024 - 256) / STAGE)));
    const size_t smem = 1024 + static_cast<size_t>(stages) * STAGE + 256;
    auto kern = tc_dst_gemm_persistent<TIn, TILE_N, OUT, SPLIT>;
    KKT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    int dev = 0, sms = 0;
    KKT_CUDA_TRY(cudaGetDevice(&dev));
    KKT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long grid = std::min<long long>(tiles, sms);
    kern<<<static_cast<unsigned>(grid), kPersistThreads, smem, st>>>(a, b, alo, blo, p, stages);
  } else {
    const size_t smem = 1024 + kStages * STAGE + 256;
    auto kern = tc_dst_gemm_kernel<TIn, TILE_N, OUT, SPLIT>;
    KKT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    kern<<<static_cast<unsigned>(tiles), 128, smem, st>>>(a, b, alo, blo, p);
  }
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

}  // namespace

// Round-to-nearest-even of a double to BF16 (8 significant bits), as a bit pattern.
uint16_t bf16_bits_rne(double v) {
  if (v == 0.0 || !std::isfinite(v)) {
    const float f = static_cast<float>(v);
    uint32_t b;
    std::memcpy(&b, &f, 4);
    return static_cast<uint16_t>(b >> 16);
  }
  int e = 0;
  const double m = std::frexp(v, &e);                 // v = m 2^e, 0.5 <= |m| < 1
  const double r = std::nearbyint(m * 256.0) / 256.0;  // 8 significant bits, ties to even
  const float f = static_cast<float>(std::ldexp(r, e)); // exact in FP32
  uint32_t b;
  std::memcpy(&b, &f, 4);
  return static_cast<uint16_t>(b >> 16);
}

// Padded transform size used by the tensor-core path: n - 1 rounded up to a multiple of 128.
int tc_padded_size(int n) { return ((n - 1 + 127) / 128) * 128; }

// hi / lo parts of a double in the operand type, as raw bits
void split_host(double v, int bf16, uint8_t* hi, uint8_t* lo) {
  if (bf16) {
    const uint16_t h = bf16_bits_rne(v);
    uint32_t hb = static_cast<uint32_t>(h) << 16;
    float hf;
    std::memcpy(&hf, &hb, 4);
    const uint16_t l = bf16_bits_rne(v - static_cast<double>(hf));
    std::memcpy(hi, &h, 2);
    std::memcpy(lo, &l, 2);
  } else {
    const float f = static_cast<float>(v);
    uint32_t b;
    std::memcpy(&b, &f, 4);
    b = (b + 0x1000u) & 0xFFFFE000u;
    float hf;
    std::memcpy(&hf, &b, 4);
    const float lf = static_cast<float>(v - static_cast<double>(hf));
    std::memcpy(hi, &hf, 4);
    std::memcpy(lo, &lf, 4);
  }
}

int tc_plan_create(TcPlan& t, int n, int slices, int bf16) {
  t = TcPlan();
  t.n = n;
  t.P = tc_padded_size(n);
  t.slices = slices;
  t.bf16 = bf16;
  const int P = t.P, M = n - 1;
  const int eb = bf16 ? 2 : 4;
  t.tile_n = P % 256 == 0 ? 256 : 128;
  const size_t plane = static_cast<size_t>(P) * P;
  const size_t elems = plane * slices;
  // Q: orthonormal DST-I matrix, zero padded
  std::vector<double> q(plane, 0.0);
  const double pi = 3.14159265358979323846, sc = std::sqrt(2.0 / n);
  for (int j = 0; j < M; ++j)
    for (int k = 0; k < M; ++k) q[static_cast<size_t>(j) * P + k] = sc * std::sin(pi * (j + 1.0) * (k + 1.0) / n);
  std::vector<uint8_t> qh(plane * eb), ql(plane * eb);
  for (size_t e = 0; e < plane; ++e) split_host(q[e], bf16, qh.data() + eb * e, ql.data() + eb * e);
  KKT_CUDA_TRY(cudaMalloc(&t.q, plane * eb));
  KKT_CUDA_TRY(cudaMalloc(&t.q_lo, plane * eb));
  KKT_CUDA_TRY(cudaMemcpy(t.q, qh.data(), plane * eb, cudaMemcpyHostToDevice));
  KKT_CUDA_TRY(cudaMemcpy(t.q_lo, ql.data(), plane * eb, cudaMemcpyHostToDevice));
  KKT_CUDA_TRY(cudaMalloc(&t.x0, elems * eb));
  KKT_CUDA_TRY(cudaMalloc(&t.x0_lo, elems * eb));
  KKT_CUDA_TRY(cudaMalloc(&t.x1, elems * eb));
  KKT_CUDA_TRY(cudaMalloc(&t.x1_lo, elems * eb));
  KKT_CUDA_TRY(cudaMalloc(&t.yin, elems * eb));
  KKT_CUDA_TRY(cudaMalloc(&t.yin_lo, elems * eb));
  KKT_CUDA_TRY(cudaMalloc(&t.rhat, elems * sizeof(float)));
  KKT_CUDA_TRY(cudaMalloc(&t.err, sizeof(int)));
  KKT_CUDA_TRY(cudaMemset(t.err, 0, sizeof(int)));
  t.bytes = 2 * plane * eb + 6 * elems * eb + elems * sizeof(float) + sizeof(int);
  const long long rows = static_cast<long long>(slices) * P;
  KKT_TRY(make_map(&t.map_q, t.q, eb, P, P, t.tile_n));
  KKT_TRY(make_map(&t.map_q_lo, t.q_lo, eb, P, P, t.tile_n));
  KKT_TRY(make_map(&t.map_x0, t.x0, eb, rows, P, kTileM));
  KKT_TRY(make_map(&t.map_x0_lo, t.x0_lo, eb, rows, P, kTileM));
  KKT_TRY(make_map(&t.map_x1, t.x1, eb, rows, P, kTileM));
  KKT_TRY(make_map(&t.map_x1_lo, t.x1_lo, eb, rows, P, kTileM));
  KKT_TRY(make_map(&t.map_yin, t.yin, eb, rows, P, kTileM));
  KKT_TRY(make_map(&t.map_yin_lo, t.yin_lo, eb, rows, P, kTileM));
  return KKT_OK;
}

void tc_plan_destroy(TcPlan& t) {
  cudaFree(t.q);
  cudaFree(t.q_lo);
  cudaFree(t.x0);
  cudaFree(t.x0_lo);
  cudaFree(t.x1);
  cudaFree(t.x1_lo);
  cudaFree(t.yin);
  cudaFree(t.yin_lo);
  cudaFree(t.rhat);
  cudaFree(t.err);
  t = TcPlan();
}

// One transform pass: out = per-slice transpose of (in-map rows) x Q. split: use the lo parts of
// the input (x0_lo / x1_lo) and of Q as well (forward transforms).
int tc_gemm(const TcPlan& t, int which_in, int out_mode, void* out, int valid, cudaStream_t st, bool split,
            void* out_lo) {
  const CUtensorMap& a = which_in == 0 ? t.map_x0 : (which_in == 1 ? t.map_x1 : t.map_yin);
  const CUtensorMap& alo = which_in == 0 ? t.map_x0_lo : (which_in == 1 ? t.map_x1_lo : t.map_yin_lo);
  TcParams p;
  p.P = t.P;
  p.slices = t.slices;
  p.valid = valid;
  p.out = out;
  p.out_lo = out_lo;
  p.err = t.err;
#define KKT_TC_CASE(TIN, TN, OM, SP)                                                       \
  if (t.tile_n == TN && out_mode == OM && split == SP)                                      \
    return launch_gemm<TIN, TN, OM, SP>(a, t.map_q, alo, t.map_q_lo, p, st);
#define KKT_TC_TYPE(TIN)                                                                   \
  KKT_TC_CASE(TIN, 256, kOutF32, true) KKT_TC_CASE(TIN, 256, kOutSplit, true)              \
  KKT_TC_CASE(TIN, 256, kOutBF16, true) KKT_TC_CASE(TIN, 128, kOutBF16, true)               \
  KKT_TC_CASE(TIN, 256, kOutF64, true) KKT_TC_CASE(TIN, 128, kOutF64, true)                 \
  KKT_TC_CASE(TIN, 256, kOutBF16, false) KKT_TC_CASE(TIN, 256, kOutF32, false)             \
  KKT_TC_CASE(TIN, 256, kOutF64, false)                                                     \
  KKT_TC_CASE(TIN, 128, kOutF32, true) KKT_TC_CASE(TIN, 128, kOutSplit, true)              \
  KKT_TC_CASE(TIN, 128, kOutBF16, false) KKT_TC_CASE(TIN, 128, kOutF32, false)             \
  KKT_TC_CASE(TIN, 128, kOutF64, false)
  if (t.bf16) {
    KKT_TC_TYPE(__nv_bfloat16)
  } else {
    KKT_TC_TYPE(float)
  }
#undef KKT_TC_TYPE
#undef KKT_TC_CASE
  return set_error(KKT_ERR_UNSUPPORTED, "tensor-core transform: unsupported output mode");
}

int tc_pack(const TcPlan& t, const double* in, int valid, cudaStream_t st) {
  const long long total = static_cast<long long>(t.slices) * t.P * t.P;
  const int tb = 256;
  if (t.slices > 65535) return set_error(KKT_ERR_UNSUPPORTED, "too many time slices for the pack grid");
  if (t.P % 2) return set_error(KKT_ERR_UNSUPPORTED, "odd padded transform size");
  const dim3 grid((t.P / 2 + tb - 1) / tb, t.P, t.slices);
  ProfScope ps(KKT_K_PACK, st, 0.0, 8.0 * t.slices * static_cast<double>(valid) * valid + 2.0 * (t.bf16 ? 2.0 : 4.0) * total);
  if (t.bf16)
    pack_kernel<__nv_bfloat16><<<grid, tb, 0, st>>>(in, static_cast<__nv_bfloat16*>(t.x0),
                                                     static_cast<__nv_bfloat16*>(t.x0_lo), t.P, valid);
  else
    pack_kernel<float><<<grid, tb, 0, st>>>(in, static_cast<float*>(t.x0), static_cast<float*>(t.x0_lo), t.P,
                                            valid);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

// Reads (and clears) the pipeline-timeout flag the transform kernels set when a bounded
// mbarrier wait ran out; a set flag is reported once as KKT_ERR_TIMEOUT.
int tc_check(const TcPlan& t, cudaStream_t st) {
  int e = 0;
  KKT_CUDA_TRY(cudaMemcpyAsync(&e, t.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  KKT_CUDA_TRY(cudaStreamSynchronize(st));
  if (e) {
    KKT_CUDA_TRY(cudaMemsetAsync(t.err, 0, sizeof(int), st));
    return set_error(KKT_ERR_TIMEOUT, "a tensor-core transform timed out waiting on its pipeline");
  }
  return KKT_OK;
}

int tc_set_flag(const TcPlan& t) {
  const int one = 1;
  KKT_CUDA_TRY(cudaMemcpy(t.err, &one, sizeof(int), cudaMemcpyHostToDevice));
  return KKT_OK;
}

namespace {

// ---- FP64-accurate sine transforms on the tensor cores ---------------------------------
//
// The orthonormal DST-I of a line x (n - 1 points) is y_c = sum_k x_k Q[k][c]. Following the
// error-free splitting of Ozaki, Ogita, Oishi and Rump ("Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its applications",
// Numer. Algorithms 59, 2012), both operands are cut into digits that the tensor cores multiply
// exactly:
//   x = 2^E_r sum_{i=1..6} a_i 2^(-8i),  Q[k][c] = 2^G_c sum_{j=1..6} b_j 2^(-8j),
// with E_r one above the exponent of line r's largest entry (so |x| < 2^(E_r - 1)), G_c the same
// for column c, and a_i, b_j balanced signed digits: the base-256 digits, less 128, of the
// 48-bit fixed-point value plus 128 in every digit position, so |a_i| <= 128 (the leading digit
// reaches 128 only at the top of its range). Each digit plane a_i 2^(-8i) is exact in BF16. A
// product plane sum_k a_i b_j 2^(-8(i+j)) is a multiple of 2^(-8L) (L = i + j) of magnitude
// at most 2^14 * 256 * 2^(-8L), so up to four products of one level accumulate exactly in FP32
// (4 * 2^22 = 2^24). Levels L = 2..5 (1, 2, 3 and 4 products) each get their own exact TMEM
// accumulator; levels 6 and 7 (11 products, at most 2^-32 of the result) share one accumulator,
// which the tensor core's FP32 accumulation rounds (measured: its error grows with the number
// of accumulation steps like a truncation, 2^-49 of the result here), and levels 8 and above
// (about 2^-46 of the result) are dropped: 21 BF16 products per tile instead of 36. The
// epilogue turns the five accumulators into one 64-bit integer in units of 2^-48 (exact for
// levels 2..5) and rounds it once to FP64: y = 2^(E_r + G_c - 48) T.
//
// Kernel: persistent and warp-specialised like the reduced-precision transform. Warp 0 lane 0
// streams, with TMA, the 6 digit planes of a 128-line x 32-K chunk of the input and the 6
// planes of the matching N-column x 32-K chunk of Q (64-byte rows, 64B swizzle) through a
// shared-memory ring; warp 1 lane 0 issues the 21 products x 2 K-steps per chunk into the five
// accumulators (5 x N TMEM columns); warps 2-9 fold the accumulators into 64-bit integers,
// release them to the next tile's MMAs, then round and store the tile, transposed per slice as
// the next pass reads it. N is 96 for 256-point padding (five accumulators take 480 of the 512
// TMEM columns; three tiles cover 288 columns, the last 32 discarded) and 64 otherwise: the
// wider tile does 1.5x the work per MMA instruction and re-reads each line's planes three
// times instead of four (measured: 0.64 against 0.77 ms per GEMM pass at 256 x 256, Nt = 1024).
constexpr int kOzN = 64;                          // output columns per tile (P = 64, 128)
constexpr int kOzNWide = 96;                      // the same for P = 256 (three tiles of 96 cover 288)
constexpr int kOzAcc = 5;                         // accumulators: levels 2, 3, 4, 5 and 6-7
constexpr int kOzProducts = kOzDigits * (kOzDigits + 1) / 2;

// Accumulator of the product of digit planes i and j (0-based): level L = i + j + 2.
__host__ __device__ constexpr int oz_acc(int i, int j) { return i + j < 4 ? i + j : 4; }

constexpr int kOzChunkBytes = 64;                 // K bytes per chunk row (32 BF16, 64B swizzle)
constexpr int kOzABytes = kTileM * kOzChunkBytes; // one digit plane: 128 lines x 32 K
constexpr int kOzEpiWarps = 8;                    // two per TMEM lane quadrant, N / 2 columns each
constexpr int kOzThreads = 64 + 32 * kOzEpiWarps;
// Per tile width N: one digit plane of Q is N columns x 32 K; a stage holds every plane of a
// chunk (72 KB at N = 64, 84 KB at N = 96), three stages at N = 64 and two at N = 96.
template <int N>
struct OzTile {
  static constexpr int kBBytes = N * kOzChunkBytes;
  static constexpr int kStageBytes = kOzDigits * (kOzABytes + kBBytes);
  static constexpr int kStages = N == kOzN ? 3 : 2;
  static constexpr size_t kSmem = 1024 + kStages * kStageBytes + 256;
  static_assert(kOzAcc * N <= 512, "TMEM: five accumulators of N columns");
  static_assert(kSmem <= 227 * 1024, "shared memory");
};
constexpr unsigned long long kOzBias = 0x808080808080ull;   // 128 in each of the six digit positions

struct OzParams {
  int P;              // padded line length (multiple of 64, at most 256)
  int M;              // points per line
  long long rows;     // lines
  int rows_pad;       // lines rounded up to 128
  const int* xexp;
  const int* qexp;
  double* out;        // [slices][M][M]; line r = s M + j, column c -> out[(s M + c) M + j]
  int* err;
};

// |v| 2^(48 - E) truncated to an integer, E = emax - 1021 (emax: the line's largest biased
// exponent): m >> (emax - e + 6), below 2^47.
__host__ __device__ inline unsigned long long oz_fixed(unsigned long long bits, int emax) {
  const int e = static_cast<int>((bits >> 52) & 0x7FF);
  if (e == 0) return 0;   // zero (subnormals flushed)
  const unsigned long long m = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = emax - e + 6;
  return sh >= 64 ? 0ull : m >> sh;
}

// The biased fixed-point value U = 128 in each digit position + sign * F (0 < U < 2^48 + 2^40).
__host__ __device__ inline unsigned long long oz_biased(unsigned long long bits, int emax) {
  const unsigned long long F = oz_fixed(bits, emax);
  return (bits >> 63) ? kOzBias - F : kOzBias + F;
}

// Balanced digit i (1-based) of U: -128..127 (the leading one up to 128).
__host__ __device__ inline int oz_digit(unsigned long long U, int i) {
  return i == 1 ? static_cast<int>(U >> 40) - 128
                : static_cast<int>((U >> (48 - kOzDigitBits * i)) & 255ull) - 128;
}

// BF16 bit pattern of d 2^(-8 level), |d| <= 128 (host side: the digit planes of Q)
inline uint16_t oz_digit_bf16(int d, int level) {
  if (d == 0) return 0;
  const unsigned a = static_cast<unsigned>(d < 0 ? -d : d), sign = d < 0 ? 1u : 0u;
  const int p = 31 - __builtin_clz(a);
  return static_cast<uint16_t>((sign << 15) | (static_cast<unsigned>(p - kOzDigitBits * level + 127) << 7) |
                               ((a << (7 - p)) & 0x7Fu));
}

// FP32 bit pattern of d 2^(-8i) (|d| <= 128, i = 1..6) in two FP32 operations: the float with
// exponent 23 - 8i and fraction bits |d| is 2^(23-8i) + |d| 2^(-8i), and subtracting 2^(23-8i)
// leaves |d| 2^(-8i) exactly. Its upper 16 bits are the BF16 digit (at most 8 significant bits:
// no rounding).
__device__ __forceinline__ uint32_t oz_digit_f32(int d, int i) {
  const uint32_t base = static_cast<uint32_t>(150 - kOzDigitBits * i) << 23;
  const unsigned a = static_cast<unsigned>(d < 0 ? -d : d);
  const float v = __uint_as_float(base | a) - __uint_as_float(base);
  return __float_as_uint(v) | (d < 0 ? 0x80000000u : 0u);
}

// One warp per line: the line's largest exponent, then its digit planes (EPL = P / 32
// consecutive elements per lane, one 4-, 8- or 16-byte store per plane) and E_r. The line is
// read coalesced (lane l: elements l, l + 32, ...) and regrouped through shared memory (one
// padding word per 8, so that the regrouping reads conflict at most 2-way).
template <int EPL>
__global__ void __launch_bounds__(256) oz_split_kernel(const double* __restrict__ in, long long rows, int M, int P,
                                                       int rows_pad, uint16_t* __restrict__ xs, int* __restrict__ xexp) {
  __shared__ unsigned long long buf[8][32 * EPL + 4 * EPL];
  const long long r = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
  if (r >= rows) return;   // uniform per warp
  const double* row = in + r * M;
  int emax = 0;
#pragma unroll
  for (int t = 0; t < EPL; ++t) {
    const int k = t * 32 + lane;
    const unsigned long long bits = k < M ? static_cast<unsigned long long>(__double_as_longlong(row[k])) : 0ull;
    emax = max(emax, static_cast<int>((bits >> 52) & 0x7FF));
    buf[wb][k + (k >> 3)] = bits;
  }
  for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  __syncwarp();
  unsigned long long b[EPL];
#pragma unroll
  for (int t = 0; t < EPL; ++t) {
    const int k = lane * EPL + t;
    b[t] = buf[wb][k + (k >> 3)];
  }
  unsigned long long U[EPL];
#pragma unroll
  for (int t = 0; t < EPL; ++t) U[t] = oz_biased(b[t], emax);
#pragma unroll
  for (int i = 1; i <= kOzDigits; ++i) {
    uint32_t w[EPL / 2];
#pragma unroll
    for (int t = 0; t < EPL; t += 2)   // upper halves of two FP32 patterns: two BF16 digits in one word
      w[t / 2] = __byte_perm(oz_digit_f32(oz_digit(U[t], i), i), oz_digit_f32(oz_digit(U[t + 1], i), i), 0x7632);
    uint16_t* dst = xs + (static_cast<long long>(i - 1) * rows_pad + r) * P + lane * EPL;
    if constexpr (EPL == 8) {
      *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    } else if constexpr (EPL == 4) {
      *reinterpret_cast<uint2*>(dst) = make_uint2(w[0], w[1]);
    } else {
      *reinterpret_cast<unsigned*>(dst) = w[0];
    }
  }
  if (lane == 0) xexp[r] = emax ? emax - 1021 : 0;
}

// y = T 2^k rounded once to FP64 (one int64 -> FP64 conversion, then the exponent added to the
// bit pattern; zero, and results outside the normal range, handled branch-free).
__device__ __forceinline__ double oz_to_double(long long T, int k) {
  const long long b = __double_as_longlong(__ll2double_rn(T));
  const long long sgn = b & static_cast<long long>(0x8000000000000000ull);
  const int e = static_cast<int>((b >> 52) & 0x7FF) + k;
  long long r = b + (static_cast<long long>(k) << 52);
  r = e <= 0 ? sgn : r;                              // below the normal range: signed zero
  r = e >= 2047 ? (sgn | 0x7FF0000000000000ll) : r;  // above it: infinity
  r = T == 0 ? 0ll : r;
  return __longlong_as_double(r);
}

template <int N>
__global__ void __launch_bounds__(kOzThreads, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmQ, OzParams p) {
  constexpr int kOzBBytes = OzTile<N>::kBBytes, kOzStageBytes = OzTile<N>::kStageBytes;
  constexpr int kOzStages = OzTile<N>::kStages, HALF = N / 2;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // stage st: planes A_0..A_5 (kOzABytes each), then B_0..B_5 (kOzBBytes each)
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kOzStages * kOzStageBytes);
  uint64_t* empty = full + kOzStages;
  uint64_t* t_full = empty + kOzStages;
  uint64_t* t_empty = t_full + 1;          // [kOzAcc]: accumulator a drained by the epilogue
  uint64_t* done = t_empty + kOzAcc;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  constexpr int KCHUNK = kOzChunkBytes / 2;             // 32 BF16 of K per chunk
  constexpr int K_STEPS = KCHUNK / 16;                  // 2 MMAs of K = 16 per chunk and product
  constexpr uint32_t IDESC = instr_desc<__nv_bfloat16, N>();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nct = (p.P + N - 1) / N, nchunks = p.P / KCHUNK;
  const long long ntiles = static_cast<long long>(p.rows_pad / kTileM) * nct;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kOzStages; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, 1);
    }
    mbar_init(t_full, 1);
    for (int a = 0; a < kOzAcc; ++a) mbar_init(t_empty + a, kOzEpiWarps);
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  long long issued = 0;   // producer: chunks whose copies were issued
  if (warp == 0) {
    if (lane == 0) {
      long long g = 0;
      for (long long tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x) {
        const int rt = static_cast<int>(tile / nct), ct = static_cast<int>(tile % nct);
        for (int c = 0; c < nchunks; ++c, ++g) {
          const int st = static_cast<int>(g % kOzStages);
          if (g >= kOzStages && !mbar_wait(empty + st, static_cast<uint32_t>(((g / kOzStages) & 1) ^ 1))) {
            *abort_flag = 1;
            break;
          }
          if (*abort_flag) break;
          uint8_t* sst = smem + st * kOzStageBytes;
          mbar_expect_tx(full + st, kOzStageBytes);
          for (int i = 0; i < kOzDigits; ++i)
            tma_load_2d(sst + i * kOzABytes, &tmX, c * KCHUNK, i * p.rows_pad + rt * kTileM, full + st);
          for (int j = 0; j < kOzDigits; ++j)
            tma_load_2d(sst + kOzDigits * kOzABytes + j * kOzBBytes, &tmQ, c * KCHUNK, j * p.P + ct * N, full + st);
          issued = g + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      long long g = 0;
      int lt = 0;
      for (long long tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x, ++lt) {
        for (int c = 0; c < nchunks; ++c, ++g) {
          const int st = static_cast<int>(g % kOzStages);
          if (!mbar_wait(full + st, static_cast<uint32_t>((g / kOzStages) & 1))) {
            *abort_flag = 1;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint8_t* sst = smem + st * kOzStageBytes;
          const uint8_t* sbq = sst + kOzDigits * kOzABytes;
          if (c == 0) {
            // the tile's first chunk, level by level: accumulator a is overwritten only after
            // the epilogue has drained it from the previous tile (its own barrier), so these
            // MMAs overlap the previous tile's epilogue
#pragma unroll
            for (int a = 0; a < kOzAcc; ++a) {
              if (lt >= 1 && !mbar_wait(t_empty + a, static_cast<uint32_t>((lt & 1) ^ 1))) {
                *abort_flag = 1;
                break;
              }
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
              const uint32_t tacc = tmem + static_cast<uint32_t>(a * N);
              bool first = true;
#pragma unroll
              for (int i = 0; i < kOzDigits; ++i)
#pragma unroll
                for (int j = 0; j + i < kOzDigits; ++j) {
                  if (oz_acc(i, j) != a) continue;
                  const uint64_t da = smem_desc64(sst + i * kOzABytes), db = smem_desc64(sbq + j * kOzBBytes);
#pragma unroll
                  for (int kk = 0; kk < K_STEPS; ++kk)
                    MmaKind<__nv_bfloat16>::mma(tacc, da + 2ull * kk, db + 2ull * kk, IDESC, (first && kk == 0) ? 0u : 1u);
                  first = false;
                }
            }
            if (*abort_flag) break;
          } else {
#pragma unroll
            for (int i = 0; i < kOzDigits; ++i) {
              const uint64_t da = smem_desc64(sst + i * kOzABytes);
#pragma unroll
              for (int j = 0; j + i < kOzDigits; ++j) {
                const uint64_t db = smem_desc64(sbq + j * kOzBBytes);
                const uint32_t tacc = tmem + static_cast<uint32_t>(oz_acc(i, j) * N);
#pragma unroll
                for (int kk = 0; kk < K_STEPS; ++kk) MmaKind<__nv_bfloat16>::mma(tacc, da + 2ull * kk, db + 2ull * kk, IDESC, 1u);
              }
            }
          }
          // this stage is free once its MMAs complete
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                       ::"r"(smem_u32(empty + st)) : "memory");
        }
        if (*abort_flag) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(smem_u32(t_full)) : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   ::"r"(smem_u32(done)) : "memory");
    }
  } else {
    // epilogue warps 2..9: warp w reads TMEM lanes 32 (w % 4) .. + 31 (the tile's lines) and
    // the half (w - 2) / 4 of the tile's N columns
    const int quad = warp & 3, half = (warp - 2) >> 2;
    int lt = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++lt) {
      if (*abort_flag) break;
      if (!mbar_wait(t_full, static_cast<uint32_t>(lt & 1))) {
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int rt = static_cast<int>(tile / nct), ct = static_cast<int>(tile % nct);
      const long long r = static_cast<long long>(rt) * kTileM + quad * 32 + lane;
      const bool row_ok = r < p.rows;
      const unsigned ru = static_cast<unsigned>(row_ok ? r : 0);
      const unsigned sl = ru / static_cast<unsigned>(p.M), jj = ru - sl * static_cast<unsigned>(p.M);
      const int er = row_ok ? p.xexp[r] : 0;
      double* obase = p.out + static_cast<long long>(sl) * p.M * p.M + jj;
      const uint32_t tbase = tmem + (static_cast<uint32_t>(quad * 32) << 16);
      // phase 1: the warp's N / 2 columns as 64-bit integers T in units of 2^-48, one accumulator
      // at a time, each released to the next tile's MMAs as soon as it is folded in. The exact
      // accumulators hold n 2^(-8L) with integer |n| <= 2^24 (levels L = 2..5), so
      // n = rint(acc 2^(8L)) is exact (a power-of-two product and an FP32 -> int32 conversion);
      // the tail (levels 6 and 7) is rounded to units of 2^-48. Horner's rule from level 2 on,
      // T = 256 T + n, gives T = sum_L n_L 2^(8(6 - L)) + tail (|T| < 2^55).
      long long T[HALF];
#pragma unroll
      for (int t = 0; t < HALF; ++t) T[t] = 0;
#pragma unroll
      for (int a = 0; a < kOzAcc; ++a) {
        const float scale = a == 0 ? 0x1p16f : a == 1 ? 0x1p24f : a == 2 ? 0x1p32f : a == 3 ? 0x1p40f : 0x1p48f;
#pragma unroll
        for (int g8 = 0; g8 < HALF / 8; ++g8) {
          uint32_t v[8];
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                       : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                       : "r"(tbase + static_cast<uint32_t>(a * N + half * HALF + g8 * 8)));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int t = 0; t < 8; ++t)
            T[g8 * 8 + t] = T[g8 * 8 + t] * 256 + __float2int_rn(__uint_as_float(v[t]) * scale);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(t_empty + a)) : "memory");
      }
      // phase 2: round to FP64 with the line's and the columns' exponents, store transposed
#pragma unroll
      for (int t = 0; t < HALF; ++t) {
        const int c = ct * N + half * HALF + t;   // (the same column in every lane: a broadcast load)
        if (row_ok && c < p.M) obase[static_cast<long long>(c) * p.M] = oz_to_double(T[t], er + __ldg(p.qexp + c) - 48);
      }
    }
  }
  __syncwarp();
  if (!mbar_wait(done, 0)) *abort_flag = 1;
  __syncthreads();
  if (*abort_flag) {
    if (threadIdx.x == 0) atomicExch(p.err, 1);
    // let this CTA's copies land before its shared memory is released (only the last
    // kOzStages issued chunks can still be in flight)
    if (warp == 0 && lane == 0) {
      for (long long c = issued > kOzStages ? issued - kOzStages : 0; c < issued; ++c)
        mbar_wait(full + static_cast<int>(c % kOzStages), static_cast<uint32_t>((c / kOzStages) & 1));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

int oz_split(const OzPlan& o, const double* in, cudaStream_t st) {
  const long long threads = o.rows * 32;
  const unsigned grid = static_cast<unsigned>((threads + 255) / 256);
  ProfScope ps(KKT_K_DST, st, 0.0, 8.0 * o.rows * o.M + 2.0 * kOzDigits * static_cast<double>(o.rows) * o.P);
  uint16_t* xs = static_cast<uint16_t*>(o.xs);
  if (o.P == 256) oz_split_kernel<8><<<grid, 256, 0, st>>>(in, o.rows, o.M, o.P, o.rows_pad, xs, o.xexp);
  else if (o.P == 128) oz_split_kernel<4><<<grid, 256, 0, st>>>(in, o.rows, o.M, o.P, o.rows_pad, xs, o.xexp);
  else oz_split_kernel<2><<<grid, 256, 0, st>>>(in, o.rows, o.M, o.P, o.rows_pad, xs, o.xexp);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

template <int N>
int oz_gemm_launch(const OzPlan& o, double* out, unsigned grid, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    KKT_CUDA_TRY(cudaFuncSetAttribute(oz_gemm_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(OzTile<N>::kSmem)));
    attr = true;
  }
  OzParams p{o.P, o.M, o.rows, o.rows_pad, o.xexp, o.qexp, out, o.err};
  oz_gemm_kernel<N><<<grid, kOzThreads, OzTile<N>::kSmem, st>>>(o.map_x, o.map_q, p);
  KKT_CUDA_TRY(cudaGetLastError());
  return KKT_OK;
}

int oz_gemm(const OzPlan& o, double* out, cudaStream_t st) {
  int dev = 0, sms = 0;
  KKT_CUDA_TRY(cudaGetDevice(&dev));
  KKT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const long long ntiles = oz_tiles(o);
  const unsigned grid = static_cast<unsigned>(std::min<long long>(ntiles, sms));
  // kOzProducts BF16 digit-plane products per tile (2 rows_pad P^2 FLOP each); planes in, FP64 out
  ProfScope ps(KKT_K_DST, st, kOzProducts * 2.0 * o.rows_pad * static_cast<double>(o.P) * o.P,
               2.0 * kOzDigits * static_cast<double>(o.rows_pad) * o.P + 8.0 * static_cast<double>(o.rows) * o.M);
  return o.N == kOzNWide ? oz_gemm_launch<kOzNWide>(o, out, grid, st) : oz_gemm_launch<kOzN>(o, out, grid, st);
}

}  // namespace

int oz_plan_create(OzPlan& o, int n, int slices) {
  o = OzPlan();
  if (n < 2 || n - 1 > 255) return set_error(KKT_ERR_UNSUPPORTED, "tensor-core FP64 transform: lines of 1..255 points");
  o.n = n;
  o.M = n - 1;
  o.P = o.M <= 64 ? 64 : (o.M <= 128 ? 128 : 256);
  o.N = o.P == 256 ? kOzNWide : kOzN;
  o.slices = slices;
  o.rows = static_cast<long long>(slices) * o.M;
  if ((o.rows + kTileM - 1) / kTileM * kTileM * kOzDigits > 0x7FFFFFFFLL)
    return set_error(KKT_ERR_UNSUPPORTED, "tensor-core FP64 transform: too many lines");
  o.rows_pad = static_cast<int>((o.rows + kTileM - 1) / kTileM * kTileM);
  const int P = o.P, M = o.M;
  // Q's digit planes and column exponents (host, integer arithmetic on the FP64 entries)
  std::vector<uint16_t> qs(static_cast<size_t>(kOzDigits) * P * P, 0);
  std::vector<int> qexp(P, 0);
  const double pi = 3.14159265358979323846, scale = std::sqrt(2.0 / n);
  std::vector<double> col(M);
  for (int c = 0; c < M; ++c) {
    int emax = 0;
    for (int k = 0; k < M; ++k) {
      col[k] = scale * std::sin(pi * (k + 1.0) * (c + 1.0) / n);
      unsigned long long b;
      std::memcpy(&b, &col[k], 8);
      emax = std::max(emax, static_cast<int>((b >> 52) & 0x7FF));
    }
    qexp[c] = emax ? emax - 1021 : 0;
    for (int k = 0; k < M; ++k) {
      unsigned long long b;
      std::memcpy(&b, &col[k], 8);
      const unsigned long long U = oz_biased(b, emax);
      for (int j = 0; j < kOzDigits; ++j)
        qs[(static_cast<size_t>(j) * P + c) * P + k] = oz_digit_bf16(oz_digit(U, j + 1), j + 1);
    }
  }
  const size_t qbytes = qs.size() * 2, xbytes = static_cast<size_t>(kOzDigits) * o.rows_pad * P * 2;
  KKT_CUDA_TRY(cudaMalloc(&o.qs, qbytes));
  KKT_CUDA_TRY(cudaMalloc(&o.qexp, P * sizeof(int)));
  KKT_CUDA_TRY(cudaMalloc(&o.xs, xbytes));
  KKT_CUDA_TRY(cudaMalloc(&o.xexp, o.rows_pad * sizeof(int)));
  KKT_CUDA_TRY(cudaMalloc(&o.tmp, static_cast<size_t>(o.rows) * M * sizeof(double)));
  KKT_CUDA_TRY(cudaMalloc(&o.err, sizeof(int)));
  KKT_CUDA_TRY(cudaMemcpy(o.qs, qs.data(), qbytes, cudaMemcpyHostToDevice));
  KKT_CUDA_TRY(cudaMemcpy(o.qexp, qexp.data(), P * sizeof(int), cudaMemcpyHostToDevice));
  // padding lines and columns stay zero: the split writes only lines < rows and columns < P
  KKT_CUDA_TRY(cudaMemset(o.xs, 0, xbytes));
  KKT_CUDA_TRY(cudaMemset(o.xexp, 0, o.rows_pad * sizeof(int)));
  KKT_CUDA_TRY(cudaMemset(o.err, 0, sizeof(int)));
  o.bytes = qbytes + xbytes + P * sizeof(int) + o.rows_pad * sizeof(int) + o.rows * M * sizeof(double) + sizeof(int);
  KKT_TRY(make_map(&o.map_x, o.xs, 2, static_cast<long long>(kOzDigits) * o.rows_pad, P, kTileM, kOzChunkBytes));
  KKT_TRY(make_map(&o.map_q, o.qs, 2, static_cast<long long>(kOzDigits) * P, P, o.N, kOzChunkBytes));
  return KKT_OK;
}

void oz_plan_destroy(OzPlan& o) {
  cudaFree(o.qs);
  cudaFree(o.qexp);
  cudaFree(o.xs);
  cudaFree(o.xexp);
  cudaFree(o.tmp);
  cudaFree(o.err);
  o = OzPlan();
}

// Both directions: along x (lines = rows of each slice) into tmp, transposed per slice, then
// along the lines of tmp (the columns of the input) into out, transposed back: out = the 2D
// transform in the input's [slice][y][x] layout. in and out may be the same array.
int oz_dst2d(const OzPlan& o, const double* in, double* out, cudaStream_t st) {
  KKT_TRY(oz_split(o, in, st));
  KKT_TRY(oz_gemm(o, o.tmp, st));
  KKT_TRY(oz_split(o, o.tmp, st));
  return oz_gemm(o, out, st);
}

long long oz_tiles(const OzPlan& o) { return static_cast<long long>(o.rows_pad / kTileM) * ((o.P + o.N - 1) / o.N); }

int oz_check(const OzPlan& o, cudaStream_t st) {
  if (!o.err) return KKT_OK;
  int e = 0;
  KKT_CUDA_TRY(cudaMemcpyAsync(&e, o.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  KKT_CUDA_TRY(cudaStreamSynchronize(st));
  if (e) {
    KKT_CUDA_TRY(cudaMemsetAsync(o.err, 0, sizeof(int), st));
    return set_error(KKT_ERR_TIMEOUT, "a tensor-core FP64 transform timed out waiting on its pipeline");
  }
  return KKT_OK;
}

}  // namespace kkt
