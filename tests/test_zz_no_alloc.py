"""lbm_observables_noalloc: observables of a saved lattice without any
allocation, for callers that may not allocate device memory on their call path
(a framework operator whose memory belongs to the framework's allocator or a
fixed budget, a monitoring stage between latency-critical GPU work).  Such a
caller keeps a checkpoint in its own device memory; the call must give what
lbm_observables gives for that state, on consecutive calls that share the
library's static scratch.  This file is collected last so that a run stopping
at the first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# the tolerance of the FP64 parity tests; both calls run the same kernels on
# the same reduction grid, so the results are expected to agree exactly
RTOL = 1e-10


def _call(lib, _lib, params, dev, nbytes, fields, stream):
    out = _lib.Obs()
    ptrs = [C.c_void_p(t.data_ptr()) for t in fields]
    rc = lib.lbm_observables_noalloc(C.byref(params), C.c_void_p(dev.data_ptr()), nbytes,
                                     C.c_void_p(stream.cuda_stream), C.byref(out), *ptrs)
    _lib.check(rc)
    return out


@pytest.mark.parametrize("precision", ["f64", "f32", "f16", "f32t"])
def test_noalloc_matches_observables_on_consecutive_calls(precision):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_2071_gb300 import Cavity, _lib

    lib = _lib.load()
    nx, ny = 96, 80
    cav = Cavity(nx, ny, Ra=1e5, Da=1e-2, phi=0.6, precision=precision)
    stream = cav.stream
    for _ in range(2):  # two calls in a row, on two different states
        cav.step(500)
        ref = cav.observables(fields=True)
        blob = cav.save()
        dev = torch.frombuffer(blob, dtype=torch.uint8).to("cuda")  # caller-owned device copy
        fields = [torch.full((ny, nx), float("nan"), dtype=cav.field_dtype, device="cuda") for _ in range(4)]
        out = _call(lib, _lib, cav.params, dev, len(blob), fields, stream)
        assert out.t == ref["t"] and out.status == 0
        for k in ("nu_hot", "nu_cold", "umax", "mass", "heat"):
            assert abs(getattr(out, k) - ref[k]) <= RTOL * abs(ref[k]), k
        for name, t in zip(("ux", "uy", "T", "p"), fields):
            a = t.double().cpu().numpy()
            b = ref[name].double().cpu().numpy()
            assert np.abs(a - b).max() <= RTOL * np.abs(b).max(), name
    cav.close()


def test_noalloc_rejects_a_mismatched_checkpoint():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_2071_gb300 import Cavity, _lib, make_params

    lib = _lib.load()
    cav = Cavity(40, 32, Ra=1e5, Da=1e-2, phi=0.6, precision="f32")
    blob = cav.save()
    dev = torch.frombuffer(blob, dtype=torch.uint8).to("cuda")
    wrong = make_params(40, 33, 1e5, 1e-2, 0.6, "f32")
    out = _lib.Obs()
    rc = lib.lbm_observables_noalloc(C.byref(wrong), C.c_void_p(dev.data_ptr()), len(blob), None, C.byref(out),
                                     None, None, None, None)
    assert rc == _lib.LBM_ERR_ARG
    small = make_params(40, 32, 1e5, 1e-2, 0.6, "f32")
    rc = lib.lbm_observables_noalloc(C.byref(small), C.c_void_p(dev.data_ptr()), 100, None, C.byref(out),
                                     None, None, None, None)
    assert rc == _lib.LBM_ERR_ARG
    assert "smaller" in lib.lbm_last_error(None).decode()
    cav.close()


def test_noalloc_reports_a_nonfinite_checkpoint_as_diverged():
    # A checkpoint carries no divergence flag of the steps that made it, so the
    # call tests the state itself: a NaN planted (on the host) into one
    # population of the saved lattice makes max|u| NaN, which it reports as
    # LBM_ERR_DIVERGED with status set, not as a finite maximum.
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_2071_gb300 import Cavity, _lib

    lib = _lib.load()
    nx, ny = 40, 32
    cav = Cavity(nx, ny, Ra=1e5, Da=1e-2, phi=0.6, precision="f64")
    cav.step(50)
    blob = bytearray(cav.save())
    # B_{n-1} follows the 40-byte header: FP64 planes with a row pitch of 48 values
    arr = np.frombuffer(blob, dtype=np.float64, count=9 * 48 * ny, offset=40)
    arr.setflags(write=True)
    arr[1 * 48 * ny + 16 * 48 + 20] = np.nan  # plane 1 (east), node (20, 16)
    dev = torch.frombuffer(blob, dtype=torch.uint8).to("cuda")
    out = _lib.Obs()
    rc = lib.lbm_observables_noalloc(C.byref(cav.params), C.c_void_p(dev.data_ptr()), len(blob),
                                     C.c_void_p(cav.stream.cuda_stream), C.byref(out), None, None, None, None)
    assert rc == _lib.LBM_ERR_DIVERGED and out.status == _lib.LBM_ERR_DIVERGED
    assert out.umax != out.umax  # NaN
    # the same call on the intact state is clean again (the status word is cleared on entry)
    good = torch.frombuffer(bytearray(cav.save()), dtype=torch.uint8).to("cuda")
    rc = lib.lbm_observables_noalloc(C.byref(cav.params), C.c_void_p(good.data_ptr()), good.numel(),
                                     C.c_void_p(cav.stream.cuda_stream), C.byref(out), None, None, None, None)
    assert rc == _lib.LBM_OK and out.status == _lib.LBM_OK and out.umax == out.umax
    cav.close()
