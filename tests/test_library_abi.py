"""The C-ABI library builds for sm_103a, loads, and exports every entry point of include/kkt.h
(no GPU: no compute call is made)."""

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^\s*(?:const char\*|int|void|kkt_handle\*)\s+(kkt_\w+)\s*\(", txt, re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2305_04421_gb300 import build, kkt
    build.build()
    return kkt.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    from paper_2305_04421_gb300 import kkt
    bound = {n for n, _, _ in kkt.SIGNATURES}
    assert set(_declared()) <= bound


def test_status_strings_and_defaults(lib):
    import ctypes
    from paper_2305_04421_gb300 import kkt
    assert lib.kkt_status_string(kkt.KKT_ERR_NONFINITE) == b"non-finite value"
    opt = kkt.KKTOptions()
    assert lib.kkt_default_options(ctypes.byref(opt)) == 0
    assert (opt.precision, opt.coarse, opt.variant, opt.pou, opt.restart, opt.jhat_sign) == (0, 0, 0, 0, 30, -1)
    assert (opt.residual_norm, opt.tc_split, opt.orth, opt.basis, opt.local) == (
        kkt.NORM["l2"], 1, kkt.ORTH["mgs2"], kkt.BASIS["physical"], kkt.LOCAL["rasq"])
    assert (opt.Lx, opt.Ly, opt.coarse_solve) == (1.0, 1.0, kkt.COARSE_SOLVE["auto"])


def test_options_struct_matches_the_header():
    """The binding's option and stats structures have the header's field order and size."""
    import ctypes
    import re
    from paper_2305_04421_gb300 import kkt
    text = open(os.path.join(ROOT, "include", "kkt.h")).read()
    body = re.search(r"typedef struct kkt_options \{(.*?)\} kkt_options;", text, re.S).group(1)
    fields = []
    for line in body.splitlines():
        m = re.match(r"\s*(int|double)\s+([\w, ]+);", line)
        if m:
            fields += [f.strip() for f in m.group(2).split(",")]
    assert [f[0] for f in kkt.KKTOptions._fields_] == fields
    assert ctypes.sizeof(kkt.KKTKernelStats) == 5 * 8 * len(kkt.KERNEL_CLASSES)
    assert "KKT_K_COUNT = %d" % len(kkt.KERNEL_CLASSES) in text


@pytest.mark.parametrize("cname,pyname", [("kkt_mlp_config", "KKTMlpConfig"),
                                          ("kkt_mlp_train_stats", "KKTMlpTrainStats"),
                                          ("kkt_instance", "KKTInstance")])
def test_network_and_batch_structs_match_the_header(cname, pyname):
    import re
    from paper_2305_04421_gb300 import kkt
    text = open(os.path.join(ROOT, "include", "kkt.h")).read()
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (cname, cname), text, re.S).group(1)
    fields = []
    for line in body.splitlines():
        m = re.match(r"\s*(int|double|long long)\s+([\w, ]+);", line)
        if m:
            fields += [f.strip() for f in m.group(2).split(",")]
    assert [f[0] for f in getattr(kkt, pyname)._fields_] == fields


def test_invalid_sizes_rejected_before_any_device_call(lib):
    assert not lib.kkt_create(1, 8, 8, 1.0, 1.0, 1e-3, 2)
    assert b"nx" in lib.kkt_last_error()
    assert not lib.kkt_create(8, 8, 8, 1.0, 1.0, 1e-3, 5)
    assert b"n_sub" in lib.kkt_last_error()
    assert not lib.kkt_create(8, 8, 8, 1.0, 1.0, 0.0, 2)


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2305_04421_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, re.M), fn


def test_binding_enum_maps_match_the_header():
    """Every name-to-value map of the binding equals the header's enum of the same kind, value for
    value and complete (a reordered or missing entry would pass wrong options silently)."""
    import paper_2305_04421_gb300.kkt as kkt
    text = open(os.path.join(ROOT, "include", "kkt.h")).read()

    def enum(name):
        body = re.search(r"enum %s \{(.*?)\};" % name, text, re.S).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        return {m.group(1): int(m.group(2)) for m in re.finditer(r"(KKT_\w+)\s*=\s*(-?\d+)", body)}

    cases = [("kkt_precision", "KKT_PREC_", kkt.PREC), ("kkt_coarse", "KKT_COARSE_", kkt.COARSE),
             ("kkt_variant", "KKT_", kkt.VARIANT), ("kkt_residual_norm", "KKT_NORM_", kkt.NORM),
             ("kkt_orth", "KKT_ORTH_", kkt.ORTH), ("kkt_basis", "KKT_BASIS_", kkt.BASIS),
             ("kkt_local", "KKT_LOCAL_", kkt.LOCAL), ("kkt_coarse_solve", "KKT_COARSE_SOLVE_", kkt.COARSE_SOLVE),
             ("kkt_pou", "KKT_POU_", kkt.POU), ("kkt_staging", "KKT_STAGING_", kkt.STAGING),
             ("kkt_dst_method", "KKT_DST_", kkt.DST_METHOD)]
    for cname, prefix, pymap in cases:
        want = {k[len(prefix):].lower(): v for k, v in enum(cname).items()}
        assert want == pymap, (cname, want, pymap)
