"""Parity of the CUDA path (through the C-ABI) with the FP64 CPU oracle.

Tolerances (max over the lattice):
  FP64 path:   populations 1e-13 absolute after one step; fields 1e-10
               relative (velocity to max|u|, temperature to dT), Nu 1e-10.
  FP32 path:   one-step populations 2e-7 absolute: stored deviations stay
               below 0.5 in magnitude (the largest is w~_0 (T_h - T0) = 0.3 at
               the hot wall), FP32 rounds them to within 3e-8, and the step's
               FP32 arithmetic adds a few more roundings of that size.
  FP16 flow:   flow deviations stay below 0.0625 (|u| <~ 0.05 here), where
               half precision rounds to within 2^-16 = 1.5e-5: one-step flow
               populations 3e-5; thermal planes are FP32 (2e-7).
  Long runs (2e4 steps) accumulate rounding; the per-field bounds below are
  the measured errors with a margin of about three.
"""
import os

import numpy as np
import pytest

from oracle import Oracle, derive
import oracle.orc as orc

pytestmark = pytest.mark.gpu

# the autotuner's cache that the benchmark uses, so that full-size cases run in its launch shapes
TUNE_CACHE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1308_2071_gb300",
                          "_build", "tune_cache.txt")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def cavity(*a, **k):
    from paper_1308_2071_gb300 import Cavity

    return Cavity(*a, **k)


def np_(t):
    return t.double().cpu().numpy()


def field_errors(obs, o):
    oux, ouy, op, oT = o.macros()
    umax = max(np.abs(oux).max(), np.abs(ouy).max(), 1e-300)
    eu = max(np.abs(np_(obs["ux"]) - oux).max(), np.abs(np_(obs["uy"]) - ouy).max()) / umax
    eT = np.abs(np_(obs["T"]) - oT).max() / (o.lat.Th - o.lat.Tc)
    ep = np.abs(np_(obs["p"]) - op).max() / np.abs(op).max()
    onl, onr = o.nusselt()
    en = max(abs(obs["nu_hot"] - onl) / abs(onl), abs(obs["nu_cold"] - onr) / abs(onr))
    return eu, eT, ep, en


# ---- one-step map, every population, several tiles and ragged tails ----------

# f16: the flow values are moved onto the half-precision grid by a dithered
# rounding, whose error stays below one unit of half precision (6.1e-5 for
# |f_i - w_i rho0| < 0.125); the thermal values of its node pairs come from
# paired FP32 instructions, which round every product (no fused multiply-add)
@pytest.mark.parametrize("precision,tol_f,tol_g", [("f64", 1e-13, 1e-13), ("f32", 2e-7, 2e-7),
                                                  ("f16", 6.2e-5, 3e-7), ("f32t", 2e-7, 2e-7)])
@pytest.mark.parametrize("shape", [(17, 13), (64, 64), (131, 70), (300, 257)])
@pytest.mark.parametrize("npt", [1, 2, 3])
def test_one_step_populations(precision, tol_f, tol_g, shape, npt, nthreads):
    nx, ny = shape
    Ra, Da, phi = 1e5, 1e-2, 0.6
    cav = cavity(nx, ny, Ra=Ra, Da=Da, phi=phi, precision=precision, nodes_per_thread=npt)
    lat = derive(nx, ny, Ra=Ra, Da=Da, phi=phi)
    o = Oracle(lat)
    for n in (0, 37, 400):
        cav.step(n - cav.query()[0])
        f, g = cav.read_state()
        o.set_state(np_(f), np_(g))
        o.step(1, threads=nthreads)
        cav.step(1)
        f1, g1 = cav.read_state()
        fo, go = o.state()
        ef = np.abs(np_(f1) - fo).max()
        eg = np.abs(np_(g1) - go).max()
        assert ef < tol_f and eg < tol_g, (n, ef, eg)
    cav.close()


@pytest.mark.parametrize("precision,tol", [("f64", 1e-15), ("f32", 2e-7), ("f16", 2e-7), ("f32t", 2e-7)])
def test_initial_state_matches_oracle(precision, tol):
    # the wall rule applied to the rest state (FP32 paths round w~_j (T_w - T0))
    cav = cavity(20, 16, Ra=1e4, Da=1e-2, phi=0.6, precision=precision)
    o = Oracle(derive(20, 16, Ra=1e4, Da=1e-2, phi=0.6))
    f, g = cav.read_state()
    fo, go = o.state()
    assert np.abs(np_(f) - fo).max() < tol
    assert np.abs(np_(g) - go).max() < tol
    cav.close()


# ---- long runs of the cavity of config 1 ---------------------------------------------

@pytest.fixture(scope="module")
def oracle_c1(nthreads):
    """64^2, Ra = 1e4, Da = 1e-2, phi = 0.6, Pr = 1: states at 200 and 20000 steps."""
    o = Oracle(derive(64, 64, Ra=1e4, Da=1e-2, phi=0.6))
    snaps = {}
    for n in (200, 20000):
        o.step(n - o.t, threads=nthreads)
        snaps[n] = (o.macros(), o.nusselt())
    return snaps


class _Snap:
    def __init__(self, macros, nus, lat):
        self._m, self._n, self.lat = macros, nus, lat

    def macros(self):
        return self._m

    def nusselt(self):
        return self._n


@pytest.mark.parametrize("precision,tol_u,tol_T,tol_nu", [
    ("f64", 1e-10, 1e-10, 1e-10),
    ("f32", 2e-4, 1e-4, 1e-4),
    ("f16", 5e-3, 1e-3, 1e-3),
    ("f32t", 2e-4, 1e-4, 1e-4),
])
def test_config1_fields_and_nusselt(oracle_c1, precision, tol_u, tol_T, tol_nu):
    lat = derive(64, 64, Ra=1e4, Da=1e-2, phi=0.6)
    cav = cavity(64, 64, Ra=1e4, Da=1e-2, phi=0.6, precision=precision)
    for n in (200, 20000):
        cav.step(n - cav.query()[0])
        obs = cav.observables(fields=True)
        eu, eT, ep, en = field_errors(obs, _Snap(*oracle_c1[n], lat))
        assert eu < tol_u and eT < tol_T and en < tol_nu, (precision, n, eu, eT, ep, en)
        assert obs["status"] == 0
    cav.close()


# ---- variants of the step --------------------------------------------------------------

def test_lbgk_mode_matches_oracle(nthreads):
    lat = derive(40, 36, Ra=1e4, Da=1e-2, phi=0.6)
    tau, tauT = 1 / lat.s[7], 1 / lat.zeta[1]
    for k in range(9):
        lat.s[k] = 1 / tau
    for k in range(5):
        lat.zeta[k] = 1 / tauT
    o = Oracle(lat).step(500, threads=nthreads)
    cav = cavity(40, 36, Ra=1e4, Da=1e-2, phi=0.6, precision="f64", collision=1)
    cav.step(500)
    eu, eT, ep, en = field_errors(cav.observables(fields=True), o)
    assert max(eu, eT, ep, en) < 1e-11, (eu, eT, ep, en)


def test_second_order_adiabatic_walls_match_oracle(nthreads):
    lat = derive(40, 36, Ra=1e5, Da=1e-2, phi=0.6)
    lat.adiabatic_order = 2
    o = Oracle(lat).step(700, threads=nthreads)
    cav = cavity(40, 36, Ra=1e5, Da=1e-2, phi=0.6, precision="f64", adiabatic_order=2)
    cav.step(700)
    eu, eT, ep, en = field_errors(cav.observables(fields=True), o)
    assert max(eu, eT, ep, en) < 1e-11, (eu, eT, ep, en)


def test_brinkman_forchheimer_off_matches_oracle(nthreads):
    lat = derive(40, 40, Ra=1e5, Da=1e-3, phi=0.5)
    lat.forchheimer = 0
    o = Oracle(lat).step(600, threads=nthreads)
    cav = cavity(40, 40, Ra=1e5, Da=1e-3, phi=0.5, precision="f64", forchheimer=0)
    cav.step(600)
    eu, eT, ep, en = field_errors(cav.observables(fields=True), o)
    assert max(eu, eT, ep, en) < 1e-11, (eu, eT, ep, en)


# tolerances: (velocity, temperature, Nu); FP16 storage rounds the flow
# deviations to 2^-11 relative every step, so its velocity bound is 1e-2
@pytest.mark.parametrize("precision,tol,shape_kw", [
    ("f64", (1e-11,) * 3, {}), ("f32", (1e-4,) * 3, {}),
    ("f32", (1e-4,) * 3, dict(nodes_per_thread=2, block_x=32, block_y=4)),
    ("f16", (1e-2, 1e-3, 1e-2), dict(nodes_per_thread=2, block_x=64, block_y=2)),
])
def test_porosity_field_matches_oracle(precision, tol, shape_kw, nthreads):
    import torch

    from paper_1308_2071_gb300.inputs import perturbed_porosity

    nx, ny = 48, 40
    phi = perturbed_porosity(ny, nx, phi_bar=0.6, amplitude=0.1, corr_len=6.0, seed=5)
    lat = derive(nx, ny, Ra=1e5, Da=1e-2, phi=0.6)
    o = Oracle(lat, phi_field=phi).step(800, threads=nthreads)
    cav = cavity(nx, ny, Ra=1e5, Da=1e-2, phi=0.6, precision=precision,
                 phi_field=torch.from_numpy(phi).cuda(), **shape_kw)
    cav.step(800)
    eu, eT, ep, en = field_errors(cav.observables(fields=True), o)
    assert eu < tol[0] and eT < tol[1] and en < tol[2], (eu, eT, ep, en)


@pytest.mark.parametrize("bad", [0.0, 1.0, float("nan"), -0.2])
@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_porosity_field_outside_the_open_unit_interval_is_rejected(bad, dtype):
    # Eq. 5 needs 0 < phi < 1 in every cell (1/phi, (1 - phi)); the library
    # checks the field on the device and refuses it before anything changes.
    import torch

    from paper_1308_2071_gb300 import _lib

    nx, ny = 37, 29
    good = torch.full((ny, nx), 0.55, dtype=getattr(torch, dtype), device="cuda")
    cav = cavity(nx, ny, Ra=1e5, Da=1e-2, phi=0.6, precision="f32", phi_field=good)
    cav.step(30)
    field = good.clone()
    field[17, 23] = bad
    with pytest.raises(_lib.LbmError, match="ARG") as e:
        cav.set_porous_field(field)
    assert "1 porosity values outside (0, 1)" in str(e.value)
    assert cav.query()[0] == 30  # the handle kept its state
    cav.set_porous_field(good)
    assert cav.query()[0] == 0
    cav.close()


@pytest.mark.parametrize("precision,tol", [("f64", 1e-11), ("f32", 2e-4), ("f16", 2e-3)])
def test_lognormal_porosity_field_matches_oracle(precision, tol, nthreads):
    # the heterogeneous input of the 8192^2 workload, at 128^2 (correlation length 8)
    import torch

    from paper_1308_2071_gb300.inputs import porosity_field

    n = 128
    phi = porosity_field(n, n, phi_bar=0.6, corr_len=8.0, seed=1308)
    assert 0.3 <= phi.min() and phi.max() <= 0.9 and phi.std() > 0.05
    lat = derive(n, n, Ra=1e5, Da=1e-4, phi=0.6)
    o = Oracle(lat, phi_field=phi).step(600, threads=nthreads)
    cav = cavity(n, n, Ra=1e5, Da=1e-4, phi=0.6, precision=precision, phi_field=torch.from_numpy(phi).cuda())
    cav.step(600)
    eu, eT, ep, en = field_errors(cav.observables(fields=True), o)
    assert max(eu, eT, en) < tol, (eu, eT, ep, en)


def test_max_size_one_step_with_porosity_field(nthreads):
    # 8192^2 with the seeded log-normal field, FP32, in the launch shape the
    # autotuner picks for it (the benchmark's): every population after one step
    # from the GPU's own state, against the oracle.
    import torch

    from paper_1308_2071_gb300.inputs import porosity_field

    n = 8192
    phi = porosity_field(n, n, phi_bar=0.6, corr_len=32.0, seed=1308)
    cav = cavity(n, n, Ra=1e5, Da=1e-4, phi=0.6, precision="f32", phi_field=torch.from_numpy(phi).cuda())
    cav.tune(TUNE_CACHE)
    cav.step(40)
    f, g = cav.read_state()
    fh, gh = np_(f), np_(g)
    del f, g
    o = Oracle(derive(n, n, Ra=1e5, Da=1e-4, phi=0.6), phi_field=phi)
    o.set_state(fh, gh)
    del fh, gh
    o.step(1, threads=nthreads)
    cav.step(1)
    f1, g1 = cav.read_state()
    fo, go = o.state()
    for q in range(9):
        assert np.abs(np_(f1[q]) - fo[q]).max() < 2e-7, q
    for q in range(5):
        assert np.abs(np_(g1[q]) - go[q]).max() < 2e-7, q
    cav.close()


# ---- full size, bench launch configuration ----------------------------------------

# f16: one unit of half precision for the dithered flow values, and the paired
# FP32 instructions of its node pairs (no fused multiply-add) for the thermal ones
@pytest.mark.parametrize("precision,tol_f,tol_g", [("f32", 2e-7, 2e-7), ("f16", 6.2e-5, 3e-7)])
def test_full_size_one_step(precision, tol_f, tol_g, nthreads):
    # 4096^2 cavity of the throughput benchmark (Ra = 1e6, Da = 1e-4, phi = 0.4)
    # in the launch shape the autotuner picks for it (the benchmark's): every
    # population after one step, from the GPU's own state, vs the oracle.
    n = 4096
    cav = cavity(n, n, Ra=1e6, Da=1e-4, phi=0.4, precision=precision)
    cav.tune(TUNE_CACHE)
    cav.step(300)
    f, g = cav.read_state()
    fh, gh = np_(f), np_(g)
    del f, g
    o = Oracle(derive(n, n, Ra=1e6, Da=1e-4, phi=0.4))
    o.set_state(fh, gh)
    del fh, gh
    o.step(1, threads=nthreads)
    cav.step(1)
    f1, g1 = cav.read_state()
    fo, go = o.state()
    for q in range(9):
        assert np.abs(np_(f1[q]) - fo[q]).max() < tol_f, q
    for q in range(5):
        assert np.abs(np_(g1[q]) - go[q]).max() < tol_g, q
    cav.close()


# ---- failure detection, checkpoint ---------------------------------------------------

@pytest.mark.parametrize("precision", ["f32", "f32t"])
def test_checkpoint_resume_is_bit_exact(precision):
    a = cavity(50, 40, Ra=1e5, Da=1e-2, phi=0.6, precision=precision)
    a.step(123)
    blob = a.save()
    a.step(77)
    ref = a.observables(fields=True)
    b = cavity(50, 40, Ra=1e5, Da=1e-2, phi=0.6, precision=precision)
    b.load(blob)
    assert b.query()[0] == 123
    b.step(77)
    got = b.observables(fields=True)
    for k in ("ux", "uy", "T", "p"):
        assert np.array_equal(np_(got[k]), np_(ref[k]))
    assert got["nu_hot"] == ref["nu_hot"]


def test_planted_nan_raises_divergence_status():
    from paper_1308_2071_gb300 import _lib

    cav = cavity(40, 40, Ra=1e5, Da=1e-2, phi=0.6, precision="f32")
    cav.step(10)
    blob = cav.save()
    # the checkpoint payload is one buffer, B_{n-1}: 14 float32 planes (row
    # pitch 64 floats for nx = 40), then the 8-bit temperature frames; lbm_load's
    # step carries the NaN into B_n
    planes = 14 * 64 * 40 * 4
    payload = planes + 64 * 40
    assert len(blob) - payload == 40  # the header
    arr = np.frombuffer(blob, dtype=np.float32, count=planes // 4, offset=40)
    k = 20 * 64 + 20  # node (20, 20) of plane 0
    arr.setflags(write=True)
    arr[k] = np.nan
    cav.load(blob)
    cav.step(3)
    t, status = cav.query()
    assert status == _lib.LBM_ERR_DIVERGED
    with pytest.raises(_lib.LbmError, match="DIVERGED"):
        cav.observables()
    assert cav.observables(check=False)["status"] == _lib.LBM_ERR_DIVERGED


# ---- launch shapes and the autotuner -----------------------------------------------

@pytest.mark.parametrize("precision,tol", [("f64", 1e-15), ("f32", 1e-7), ("f16", 6.2e-5)])
@pytest.mark.parametrize("shape", [(17, 13), (131, 70)])
def test_launch_shapes_agree_to_one_rounding(precision, tol, shape):
    # The two-nodes-per-thread kernel evaluates the same formulas; the compiler
    # may fuse multiply-adds differently, so one step from the same state
    # agrees to within a rounding of the stored values (f16: one unit of half
    # precision, as the dithered rounding may go either way).
    nx, ny = shape
    ref = cavity(nx, ny, Ra=1e5, Da=1e-2, phi=0.6, precision=precision, nodes_per_thread=1)
    ref.step(200)
    blob = ref.save()
    ref.step(1)
    f0, g0 = (np_(t) for t in ref.read_state())
    for npt, bx, by in ((2, 32, 4), (2, 128, 1), (1, 64, 4), (3, 32, 4), (3, 64, 2), (3, 256, 1)):
        cav = cavity(nx, ny, Ra=1e5, Da=1e-2, phi=0.6, precision=precision, nodes_per_thread=npt,
                     block_x=bx, block_y=by)
        cav.load(blob)
        cav.step(1)
        f1, g1 = (np_(t) for t in cav.read_state())
        assert np.abs(f1 - f0).max() <= tol and np.abs(g1 - g0).max() <= tol, (npt, bx, by)
        cav.close()


def test_step_autotuner_resets_and_caches(tmp_path):
    cache = str(tmp_path / "tune.txt")
    cav = cavity(300, 200, Ra=1e5, Da=1e-2, phi=0.6, precision="f32")
    cav.step(20)
    shape = cav.tune(cache)
    assert cav.query()[0] == 0 and shape[2] in (1, 2) and shape[0] * shape[1] <= 256
    assert len(open(cache).read().splitlines()) == 1
    cav2 = cavity(300, 200, Ra=1e5, Da=1e-2, phi=0.6, precision="f32")
    assert cav2.tune(cache) == shape
    assert len(open(cache).read().splitlines()) == 1
    cav.step(40)
    cav2.step(40)
    assert np.array_equal(np_(cav.read_state()[0]), np_(cav2.read_state()[0]))


# ---- internal heat generation (Sections 4.2-4.3) and Da = infinity ------------------

@pytest.mark.parametrize("case", ["cooled", "side_heated", "no_darcy"])
def test_internal_heating_and_infinite_darcy_match_oracle(case, nthreads):
    n = 48
    if case == "cooled":  # Section 4.2 set-up: every wall at Tc, Ra = 0, Brinkman model
        kw = dict(Ra=0.0, Da=1e-2, phi=1.0, Pr=7.0, RaI=6.4e5, thermal_bc=1)
        lat = derive(n, n, Ra=0.0, Da=1e-2, phi=1.0, Pr=7.0, RaI=6.4e5, thermal_bc=1)
        lat.forchheimer = 0
        extra = dict(forchheimer=0)
    elif case == "side_heated":  # Section 4.3 set-up
        kw = dict(Ra=1e5, Da=1e-2, phi=0.4, Pr=0.7, RaI=1e7)
        lat = derive(n, n, Ra=1e5, Da=1e-2, phi=0.4, Pr=0.7, RaI=1e7)
        extra = {}
    else:  # pure fluid limit with no Darcy drag
        kw = dict(Ra=1e5, Da=float("inf"), phi=1.0, Pr=0.71)
        lat = derive(n, n, Ra=1e5, Da=float("inf"), phi=1.0, Pr=0.71)
        lat.forchheimer = 0
        extra = dict(forchheimer=0)
    o = Oracle(lat).step(700, threads=nthreads)
    cav = cavity(n, n, precision="f64", **kw, **extra)
    cav.step(700)
    obs = cav.observables(fields=True)
    eu, eT, ep, en = field_errors(obs, o)
    if case == "cooled":
        # internal heating has barely set the fluid moving after 700 steps:
        # measure the velocity error against the velocity scale U = Ma c_s
        oux, ouy, _, _ = o.macros()
        U = 0.1 / np.sqrt(3.0)
        eu = max(np.abs(np_(obs["ux"]) - oux).max(), np.abs(np_(obs["uy"]) - ouy).max()) / U
    assert max(eu, eT, ep) < 1e-11, (eu, eT, ep, en)
    assert en < 1e-10 or case == "cooled", en


# ---- the Nusselt read-back (row-parallel reduction, synchronous and asynchronous) ------

@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("shape", [(40, 31), (96, 600)])  # one block; three blocks, ragged
def test_nusselt_readback_matches_oracle(precision, tol, shape, nthreads):
    import torch

    nx, ny = shape
    cav = cavity(nx, ny, Ra=1e5, Da=1e-2, phi=0.6, precision=precision)
    o = Oracle(derive(nx, ny, Ra=1e5, Da=1e-2, phi=0.6))
    buf = torch.zeros((4, 2), dtype=torch.float64, pin_memory=True)
    for k, n in enumerate((1, 150, 151, 400)):
        cav.step(n - cav.query()[0])
        o.step(n - o.t, threads=nthreads)
        cav.nusselt_async(buf.data_ptr() + 16 * k)
        nh, nc = cav.nusselt()  # waits for the stream, so the copy above has landed
        assert (float(buf[k, 0]), float(buf[k, 1])) == (nh, nc)
        onh, onc = o.nusselt()
        assert abs(nh - onh) <= tol * abs(onh) and abs(nc - onc) <= tol * abs(onc), (n, nh, onh, nc, onc)
        obs = cav.observables()
        assert abs(obs["nu_hot"] - nh) <= 1e-12 * abs(nh)  # other summation order
    cav.close()


# ---- Nusselt numbers of every step from the step kernel (lbm_step_nusselt) ------------

# name: (nx, ny, precision, keyword arguments); "field" adds a seeded porosity field
STEP_NU_CASES = {
    "f64": (40, 31, "f64", {}),
    "f32_two_nodes": (96, 70, "f32", dict(nodes_per_thread=2, block_x=32, block_y=4)),
    "f32_one_node": (96, 70, "f32", dict(nodes_per_thread=1, block_x=64, block_y=2)),
    "f16_paired": (96, 70, "f16", dict(nodes_per_thread=2, block_x=64, block_y=2)),
    "f32t": (96, 70, "f32t", {}),
    "f32t_adiabatic_order2": (40, 36, "f32t", dict(adiabatic_order=2)),
    "f32_adiabatic_order2": (40, 36, "f32", dict(adiabatic_order=2)),
    "f64_field": (48, 40, "f64", "field"),
    "f32_field": (48, 40, "f32", "field"),
    "narrow": (7, 9, "f32", {}),  # the column sets of both walls overlap
    "cooled": (48, 48, "f64", dict(Ra=0.0, Da=1e-2, phi=1.0, Pr=7.0, RaI=6.4e5, thermal_bc=1, forchheimer=0)),
}


@pytest.mark.parametrize("case", list(STEP_NU_CASES))
def test_step_nusselt_equals_step_then_nusselt(case):
    """Every step's Nusselt numbers from the wall columns the observing step
    stores equal lbm_nusselt after lbm_step bit for bit, and the lattice is
    the same, in device and in pinned host output memory."""
    import torch

    from paper_1308_2071_gb300.inputs import perturbed_porosity

    nx, ny, precision, kw = STEP_NU_CASES[case]
    base = dict(Ra=1e5, Da=1e-2, phi=0.6, precision=precision)
    if kw == "field":
        phi = perturbed_porosity(ny, nx, phi_bar=0.6, amplitude=0.1, corr_len=6.0, seed=5)
        kw = dict(phi_field=torch.from_numpy(phi).cuda())
    base.update(kw)
    a, b = cavity(nx, ny, **base), cavity(nx, ny, **base)
    n1, n2 = 40, 17
    ref = np.array([a.step(1).nusselt() for _ in range(n1 + n2)])
    got_dev = b.step_nusselt(n1)
    host = torch.zeros((n2, 2), dtype=torch.float64, pin_memory=True)
    b.step_nusselt(n2, out=host)
    b.stream.synchronize()
    got = np.concatenate([got_dev.cpu().numpy(), host.numpy()])
    assert np.array_equal(got, ref), np.abs(got - ref).max()
    assert np.isfinite(ref).all() and a.query()[0] == b.query()[0] == n1 + n2
    assert bytes(a.save()) == bytes(b.save())
    assert b.nusselt() == tuple(ref[-1])
    a.close()
    b.close()


def test_step_nusselt_matches_oracle_series(nthreads):
    """Config 1 lattice: the per-step Nusselt series against the oracle's at
    the steps it is sampled on."""
    o = Oracle(derive(64, 64, Ra=1e4, Da=1e-2, phi=0.6))
    cav = cavity(64, 64, Ra=1e4, Da=1e-2, phi=0.6, precision="f64")
    series = cav.step_nusselt(300).cpu().numpy()
    for t in (1, 2, 50, 299, 300):
        o.step(t - o.t, threads=nthreads)
        onh, onc = o.nusselt()
        nh, nc = series[t - 1]
        assert abs(nh - onh) <= 1e-11 * abs(onh) and abs(nc - onc) <= 1e-11 * abs(onc), (t, nh, onh, nc, onc)
    cav.close()


def test_step_nusselt_rejects_pageable_output_and_bad_arguments():
    import ctypes as C

    from paper_1308_2071_gb300 import _lib

    lib = _lib.load()
    cav = cavity(32, 32, Ra=1e4, Da=1e-2, phi=0.6)
    pageable = (C.c_double * 8)()
    assert lib.lbm_step_nusselt(cav.handle, 4, C.cast(pageable, C.c_void_p)) == _lib.LBM_ERR_ARG
    assert "page-locked" in lib.lbm_last_error(cav.handle).decode()
    assert lib.lbm_step_nusselt(cav.handle, 4, None) == _lib.LBM_ERR_ARG
    assert lib.lbm_step_nusselt(cav.handle, -1, None) == _lib.LBM_ERR_ARG
    assert lib.lbm_step_nusselt(cav.handle, 0, None) == _lib.LBM_OK
    assert cav.query()[0] == 0  # nothing ran
    cav.close()


# ---- config 2 at 1024^2, a long run -----------------------------------------------------

@pytest.fixture(scope="module")
def oracle_c2_1024(nthreads):
    """1024^2, Ra = 1e6, Da = 1e-4, phi = 0.4 (the throughput benchmark's physics): the oracle
    after 2000 steps (about 2e9 node updates)."""
    o = Oracle(derive(1024, 1024, Ra=1e6, Da=1e-4, phi=0.4))
    o.step(2000, threads=nthreads)
    return o.macros(), o.nusselt()


@pytest.mark.parametrize("precision,tol_u,tol_T,tol_nu", [
    ("f64", 1e-10, 1e-10, 1e-10),
    ("f32", 1e-4, 1e-5, 1e-4),
])
def test_config2_1024_long_run_matches_oracle(oracle_c2_1024, precision, tol_u, tol_T, tol_nu):
    lat = derive(1024, 1024, Ra=1e6, Da=1e-4, phi=0.4)
    cav = cavity(1024, 1024, Ra=1e6, Da=1e-4, phi=0.4, precision=precision)
    cav.tune(TUNE_CACHE)
    cav.step(2000)
    obs = cav.observables(fields=True)
    eu, eT, ep, en = field_errors(obs, _Snap(*oracle_c2_1024, lat))
    assert eu < tol_u and eT < tol_T and en < tol_nu, (precision, eu, eT, ep, en)
    assert obs["status"] == 0
    cav.close()
