"""CPU checks of the C ABI: the library builds for sm_103a, loads without a
GPU, exports every function include/lsq.h declares, and the ctypes
structures match the C layout.  No compute call is made here."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2406_03468_gb300 as lsq

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lsq.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lsq_[A-Za-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(lsq.library_path() if os.path.exists(lsq.library_path()) else lsq._build.build())
    names = declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
        assert name in lsq.EXPORTED, name


def test_struct_layout_matches_c(tmp_path):
    prog = tmp_path / "sz.c"
    prog.write_text('#include "lsq.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(lsq_options), '
                    'sizeof(lsq_info), offsetof(lsq_options, fixed_inner), '
                    'offsetof(lsq_info, ms_total), offsetof(lsq_options, qr_wait_us), '
                    'sizeof(lsq_batch_item), offsetof(lsq_batch_item, status), '
                    'offsetof(lsq_options, sparse)); '
                    'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert int(out[0]) == ctypes.sizeof(lsq.LsqOptions)
    assert int(out[1]) == ctypes.sizeof(lsq.LsqInfo)
    assert int(out[2]) == lsq.LsqOptions.fixed_inner.offset
    assert int(out[3]) == lsq.LsqInfo.ms_total.offset
    assert int(out[4]) == lsq.LsqOptions.qr_wait_us.offset
    assert int(out[5]) == ctypes.sizeof(lsq.LsqBatchItem)
    assert int(out[6]) == lsq.LsqBatchItem.status.offset
    assert int(out[7]) == lsq.LsqOptions.sparse.offset


def test_defaults_and_validation_without_gpu():
    o = lsq.lsq_options_default(m=100, n=10)
    assert o.zeta == 8 and o.col_scale == 1 and o.max_inner == 100 and o.max_refine == 2
    assert abs(o.stop_rho - 0.4) < 1e-15 and o.stop_gamma == 10.0
    bad = lsq.lsq_options_default(m=5, n=10)          # m < n is rejected before any CUDA call
    with pytest.raises(lsq.LsqError) as e:
        lsq.lsq_plan_create(bad)
    assert e.value.status == -1
    bad = lsq.lsq_options_default(m=100, n=10, zeta=40)
    with pytest.raises(lsq.LsqError):
        lsq.lsq_plan_create(bad)


def test_build_targets_sm103a_only():
    from paper_2406_03468_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


# Each option rule of the plan's validation (run before any CUDA call): a
# violation returns LSQ_ERR_INVALID; the valid neighbour passes validation
# and, on a machine without a GPU, stops at the device query (LSQ_ERR_CUDA).
_RULES = [
    ({"m": 100, "n": 0}, {"m": 100, "n": 1}),                      # n >= 1
    ({"m": 100, "n": 10, "lda": 9}, {"m": 100, "n": 10, "lda": 10}),
    ({"m": 100, "n": 10, "d": 9}, {"m": 100, "n": 10, "d": 10}),   # n <= d
    ({"m": 100, "n": 10, "d": (1 << 24) + 1}, {"m": 100, "n": 10, "d": 1 << 24}),
    ({"m": 100, "n": 10, "d": 12, "zeta": 13}, {"m": 100, "n": 10, "d": 12, "zeta": 12}),
    ({"m": 100, "n": 10, "zeta": 33}, {"m": 100, "n": 10, "zeta": 32}),
    ({"m": 100, "n": 10, "max_inner": -1}, {"m": 100, "n": 10, "max_inner": 0}),
    ({"m": 100, "n": 10, "max_refine": 9}, {"m": 100, "n": 10, "max_refine": 8}),
    ({"m": 100, "n": 10, "max_refine": -1}, {"m": 100, "n": 10, "max_refine": 0}),
    ({"m": 2000, "n": 1025}, {"m": 2000, "n": 1024}),             # n <= LSQ_MAX_N
    ({"m": 100, "n": 10, "eta": 1.0}, {"m": 100, "n": 10, "eta": 0.99}),
    ({"m": 100, "n": 10, "eta": -0.1}, {"m": 100, "n": 10, "eta": 0.0}),
    ({"m": 100, "n": 10, "precision": 3}, {"m": 100, "n": 10, "precision": 2}),
    ({"m": 100, "n": 10, "qr_wait_us": -1}, {"m": 100, "n": 10, "qr_wait_us": 0}),
    ({"m": 100, "n": 10, "kw_stop": 2}, {"m": 100, "n": 10, "kw_stop": 1}),
    ({"m": 100, "n": 10, "nrhs": 12}, {"m": 100, "n": 10, "nrhs": 16}),   # multiple of 8
    ({"m": 1000, "n": 300, "nrhs": 8}, {"m": 1000, "n": 256, "nrhs": 8}),  # n <= 256
    ({"m": 100, "n": 10, "sparse": 2}, {"m": 100, "n": 10, "sparse": 1}),
    ({"m": 100, "n": 10, "sparse": 1, "nrhs": 8}, {"m": 100, "n": 10, "sparse": 1}),
    ({"m": 100, "n": 10, "sparse": 1, "kw_stop": 1}, {"m": 100, "n": 10, "sparse": 1}),
    ({"m": 100, "n": 10, "sparse": 1, "precision": 0}, {"m": 100, "n": 10, "sparse": 1,
                                                        "precision": 1}),
]


@pytest.mark.parametrize("bad,good", _RULES)
def test_option_rules_without_gpu(bad, good):
    import torch
    if torch.cuda.is_available():
        pytest.skip("checks the validation order on a machine without a GPU")
    with pytest.raises(lsq.LsqError) as e:
        lsq.lsq_plan_create(lsq.lsq_options_default(**bad))
    assert e.value.status == -1, (bad, lsq.lsq_last_error())
    with pytest.raises(lsq.LsqError) as e:
        lsq.lsq_plan_create(lsq.lsq_options_default(**good))
    assert e.value.status == -3, (good, lsq.lsq_last_error())


_HANDLE_ENTRIES = [
    "lsq_plan_configure", "lsq_sketch", "lsq_solve_fossils", "lsq_solve_spir",
    "lsq_solve_spir_lsqr", "lsq_solve_host", "lsq_solve_fossils_multi", "lsq_solve_complex",
    "lsq_solve_csr", "lsq_sketch_pattern", "lsq_get_sketch", "lsq_get_sketch_raw", "lsq_get_R",
    "lsq_apply_normal", "lsq_apply_normal_multi", "lsq_residual", "lsq_sketched_kw", "lsq_trsv",
    "lsq_batch_solve", "lsq_submit", "lsq_poll", "lsq_server_stats",
]


@pytest.mark.parametrize("name", _HANDLE_ENTRIES)
def test_null_handle_is_invalid(name):
    """Every entry point that takes a plan, batch or server handle returns
    LSQ_ERR_INVALID for a NULL handle (all pointer arguments NULL, sizes 0)
    before any CUDA call; the destroy calls accept NULL."""
    import ctypes
    L = lsq._lib()
    _, args = lsq.EXPORTED[name]
    vals = [0 if a in (ctypes.c_int, ctypes.c_long, ctypes.c_ulong) else None for a in args]
    assert getattr(L, name)(*vals) == -1, lsq.lsq_last_error()


def test_destroy_accepts_null():
    L = lsq._lib()
    for name in ("lsq_plan_destroy", "lsq_batch_destroy", "lsq_server_destroy"):
        getattr(L, name)(None)
