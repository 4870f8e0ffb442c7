"""Host-side checks of the C-ABI: the library builds for sm_103a, loads, exports every entry
point declared in include/nlint.h, and rejects bad arguments before touching the GPU."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "nlint.h")


def declared_symbols():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(nlint_\w+)\s*\(", txt, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1311_4120_gb300 import build as b
    b.build()
    import paper_1311_4120_gb300 as pkg
    return pkg.load_library()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("nlint_plan_create", "nlint_eval", "nlint_energy", "nlint_plan_destroy",
              "nlint_last_error", "nlint_type2", "nlint_type1", "nlint_eval_host"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    import paper_1311_4120_gb300 as pkg
    assert set(declared_symbols()) <= set(pkg.EXPORTED)


def _create(lib, **kw):
    import paper_1311_4120_gb300 as pkg
    prm = pkg.nlint_params()
    lib.nlint_params_default(ctypes.byref(prm))
    for k, v in kw.items():
        if k == "axis":
            for a in range(3):
                prm.axis[a] = v[a]
        else:
            setattr(prm, k, v)
    h = ctypes.c_void_p()
    rc = lib.nlint_plan_create_ex(ctypes.byref(prm), ctypes.byref(h))
    return rc, lib.nlint_last_error().decode()


@pytest.mark.parametrize("kw,code,word", [
    (dict(d=4), -1, "d must"),
    (dict(n=31), -1, "even"),
    (dict(n=4), -1, "even"),
    (dict(L=0.0), -1, "L must"),
    (dict(L=-2.0), -1, "L must"),
    (dict(kernel=7), -1, "kernel"),
    (dict(kernel=1, axis=(0.0, 0.0, 0.0)), -1, "axis"),
    (dict(n=2048), -5, "2048"),
    (dict(d=2, kernel=1, axis=(1.0, 0.0, 0.0), alpha=float("inf")), -1, "alpha"),
    (dict(P=100.0), -1, "P must"),
    (dict(w=40), -1, "width"),
    (dict(n_phi=63), -1, "n_phi"),
    (dict(n_theta=31, n_r=16, n_phi=32), -1, "n_theta"),
    (dict(sigma=1.1), -1, "sigma"),
    (dict(algorithm=3), -1, "algorithm"),
    (dict(algorithm=2, pu_a=-1.0), -1, "Algorithm 2"),
    (dict(algorithm=2, pu_a=float("nan")), -1, "Algorithm 2"),
    (dict(algorithm=2, P2=100.0), -1, "P2"),
    (dict(algorithm=2, d=2, pu_r0=2.0, pu_r1=1.0), -1, "pu_r0 < pu_r1"),
    (dict(fft_sched=16), -1, "fft_sched"),
    (dict(fft_sched=-1), -1, "fft_sched"),
])
def test_bad_arguments_are_rejected_before_any_gpu_work(lib, kw, code, word):
    rc, msg = _create(lib, **kw)
    assert rc == code
    assert word in msg


def test_null_arguments(lib):
    assert lib.nlint_plan_create_ex(None, None) == -1
    assert lib.nlint_eval(None, None, None, None) == -1
    assert lib.nlint_plan_info(None, None) == -1
    assert lib.nlint_plan_check(None) == -1
    assert lib.nlint_eval_host_many(None, 2, None, None, 1.0, None, None) == -1
    assert lib.nlint_autotune_batch(0, None, 1e-5, None, 0, None, None, None) == -1
    lib.nlint_plan_destroy(None)  # no-op


def test_batch_autotune_rejects_mixed_devices(lib):
    import paper_1311_4120_gb300 as pkg
    arr = (pkg.nlint_params * 2)()
    for i in range(2):
        lib.nlint_params_default(ctypes.byref(arr[i]))
        arr[i].n, arr[i].device = 32, i
    out = (pkg.nlint_params * 2)()
    assert lib.nlint_autotune_batch(2, arr, 1e-5, None, 0, out, None, None) == -1
    assert "different devices" in lib.nlint_last_error().decode()


def test_params_default(lib):
    import paper_1311_4120_gb300 as pkg
    prm = pkg.nlint_params()
    lib.nlint_params_default(ctypes.byref(prm))
    assert prm.d == 3 and prm.kernel == 0 and prm.precision == -1 and prm.device == -1
    assert prm.eps == 1e-6
    # the last fields: the ctypes mirror of the struct ends where the C struct does
    assert prm.algorithm == 1 and prm.pu_a == 0.0 and prm.pu_r0 == 0.0 and prm.P2 == 0.0
    assert prm.bin_shape == 0 and prm.fft_sched == 0
    sentinel = (ctypes.c_char * (ctypes.sizeof(prm) + 64))()
    ctypes.memset(sentinel, 0x5A, len(sentinel))
    lib.nlint_params_default(ctypes.cast(sentinel, ctypes.POINTER(pkg.nlint_params)))
    assert bytes(sentinel[ctypes.sizeof(prm):]) == b"\x5a" * 64
