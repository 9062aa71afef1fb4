"""Discrete adjoint (lbm_adjoint_step): dJ/dphi of the hot-wall mean Nusselt
number against central differences of the FP64 oracle, on single cells of
every kind (hot wall, corner, adiabatic wall, next to walls, interior, cold
wall) and along random directions."""
import numpy as np
import pytest

from oracle import Oracle, derive

pytestmark = pytest.mark.gpu

NX, NY, N, K = 40, 36, 300, 64
RA, DA, PHIBAR = 1e5, 1e-2, 0.6
CELLS = [(0, 10), (1, 10), (2, 17), (3, 3), (1, 1), (0, 0), (1, 0), (4, 35), (5, 18), (10, 18), (20, 18),
         (38, 18), (39, 18), (6, 2), (2, 6), (15, 30)]


@pytest.fixture(scope="module")
def phi():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1308_2071_gb300.inputs import perturbed_porosity

    return perturbed_porosity(NY, NX, phi_bar=PHIBAR, amplitude=0.05, corr_len=6.0, seed=11)


def j_oracle(phi, nthreads):
    o = Oracle(derive(NX, NY, Ra=RA, Da=DA, phi=PHIBAR), phi_field=phi).step(N, threads=nthreads)
    return o.nusselt()[0]


@pytest.fixture(scope="module")
def finite_differences(phi, nthreads):
    fd = []
    for (x, y) in CELLS:
        h = 1e-5 * phi[y, x]
        p = phi.copy()
        p[y, x] += h
        jp = j_oracle(p, nthreads)
        p[y, x] -= 2 * h
        jm = j_oracle(p, nthreads)
        fd.append((jp - jm) / (2 * h))
    rng = np.random.default_rng(5)
    dirs = []
    for _ in range(2):
        v = rng.standard_normal(phi.shape)
        v /= np.linalg.norm(v)
        h = 1e-5
        fd.append((j_oracle(phi + h * v, nthreads) - j_oracle(phi - h * v, nthreads)) / (2 * h))
        dirs.append(v)
    return np.array(fd), dirs, j_oracle(phi, nthreads)


@pytest.mark.parametrize("precision,tol,tol_j", [("f64", 1e-6, 1e-10), ("f32", 1e-3, 1e-4)])
def test_adjoint_matches_oracle_central_differences(phi, finite_differences, precision, tol, tol_j):
    import torch

    from paper_1308_2071_gb300 import Cavity

    fd, dirs, j0 = finite_differences
    cav = Cavity(NX, NY, Ra=RA, Da=DA, phi=PHIBAR, precision=precision, phi_field=torch.from_numpy(phi).cuda())
    J, g = cav.adjoint(N, K)
    assert abs(J - j0) <= tol_j * abs(j0)
    assert cav.query()[0] == N and abs(cav.nusselt()[0] - J) <= 1e-12 * abs(J)
    g = g.double().cpu().numpy()
    ad = [g[y, x] for (x, y) in CELLS] + [float((g * v).sum()) for v in dirs]
    ad = np.array(ad)
    err = np.linalg.norm(ad - fd) / np.linalg.norm(fd)
    assert err < tol, (err, list(zip(ad, fd)))
    cav.close()


def test_checkpoint_interval_does_not_change_the_gradient(phi):
    import torch

    from paper_1308_2071_gb300 import Cavity

    grads = []
    for k in (1, 7, 64, 1000):
        cav = Cavity(NX, NY, Ra=RA, Da=DA, phi=PHIBAR, precision="f64", phi_field=torch.from_numpy(phi).cuda())
        grads.append(cav.adjoint(120, k)[1].cpu().numpy())
        cav.close()
    for g in grads[1:]:
        assert np.array_equal(g, grads[0])


def test_adjoint_requires_a_porosity_field():
    from paper_1308_2071_gb300 import Cavity, _lib

    cav = Cavity(20, 20, Ra=1e4, Da=1e-2, phi=0.6, precision="f32")
    with pytest.raises(_lib.LbmError, match="STATE"):
        cav.adjoint(10, 5)
    cav.close()


# ---- torch.autograd.Function ------------------------------------------------------------

def test_autograd_function_gives_the_adjoint_gradient(phi, finite_differences):
    import torch

    from paper_1308_2071_gb300 import Cavity, hot_wall_nusselt

    fd, dirs, j0 = finite_differences
    cav = Cavity(NX, NY, Ra=RA, Da=DA, phi=PHIBAR, precision="f64", phi_field=torch.from_numpy(phi).cuda())
    J_ref, g_ref = cav.adjoint(N, K)
    p = torch.from_numpy(phi).cuda().requires_grad_(True)
    J = hot_wall_nusselt(p, cav, N, K)
    assert J.dim() == 0 and float(J.detach()) == J_ref  # same launches, same rounding
    (3.0 * J).backward()
    assert torch.equal(p.grad, 3.0 * g_ref)
    g = p.grad.cpu().numpy() / 3.0
    ad = np.array([g[y, x] for (x, y) in CELLS] + [float((g * v).sum()) for v in dirs])
    assert np.linalg.norm(ad - fd) / np.linalg.norm(fd) < 1e-6
    # without requires_grad it is a plain forward run
    with torch.no_grad():
        assert float(hot_wall_nusselt(p.detach(), cav, N, K)) == J_ref
    cav.close()


def test_autograd_backward_detects_a_changed_cavity(phi):
    import torch

    from paper_1308_2071_gb300 import Cavity, hot_wall_nusselt

    cav = Cavity(NX, NY, Ra=RA, Da=DA, phi=PHIBAR, precision="f32", phi_field=torch.from_numpy(phi).cuda())
    p = torch.from_numpy(phi).float().cuda().requires_grad_(True)
    J = hot_wall_nusselt(p, cav, 40, 16)
    J.backward()
    assert p.grad.dtype == torch.float32 and torch.isfinite(p.grad).all()
    p.grad = None
    J = hot_wall_nusselt(p, cav, 40, 16)
    cav.close()
    cav2 = Cavity(NX, NY, Ra=10 * RA, Da=DA, phi=PHIBAR, precision="f32", phi_field=p.detach())
    # rebinding the recorded cavity to another one with other parameters must be caught
    J.grad_fn.cavity = cav2
    with pytest.raises(RuntimeError, match="changed between forward and backward"):
        J.backward()
    cav2.close()


# ---- the sizes the gradient benchmark states ------------------------------------------

def _cells_of_every_kind(n):
    """16 cells on a square n x n cavity: the hot wall, its corners, the adiabatic
    walls, next to each wall, the interior and the cold wall."""
    m = n // 2
    return [(0, m), (0, 0), (0, n - 1), (1, m), (2, m + 3), (m, 0), (m + 5, n - 1), (m, 1), (m - 7, n - 2),
            (m, m), (n // 4, 3 * n // 4), (3 * n // 4, n // 5), (n - 2, m), (n - 1, m - 4), (n - 1, 0), (1, 1)]


def _fd_cells_and_directions(phi, nsteps, nthreads, cells, ndirs, seed):
    """Central differences of the FP64 oracle's J = Nu_hot(t_N): h = 1e-5 phi at
    single cells, h = 1e-5 along unit random directions."""
    n = phi.shape[0]

    def J(p):
        o = Oracle(derive(n, n, Ra=1e5, Da=1e-2, phi=0.6), phi_field=p).step(nsteps, threads=nthreads)
        return o.nusselt()[0]

    fd = []
    for (x, y) in cells:
        h = 1e-5 * phi[y, x]
        p = phi.copy()
        p[y, x] += h
        jp = J(p)
        p[y, x] -= 2 * h
        fd.append((jp - J(p)) / (2 * h))
    rng = np.random.default_rng(seed)
    dirs = []
    for _ in range(ndirs):
        v = rng.standard_normal(phi.shape)
        v /= np.linalg.norm(v)
        fd.append((J(phi + 1e-5 * v) - J(phi - 1e-5 * v)) / 2e-5)
        dirs.append(v)
    return np.array(fd), dirs


@pytest.fixture(scope="module")
def fd_64(nthreads):
    """64^2 cavity of the gradient benchmark's physics (Ra 1e5, Da 1e-2, porosity
    0.6 plus a smooth perturbation), 2000 steps: 16 cells and 2 directions."""
    from paper_1308_2071_gb300.inputs import perturbed_porosity

    phi = perturbed_porosity(64, 64, phi_bar=0.6, amplitude=0.05, corr_len=8.0, seed=64)
    cells = _cells_of_every_kind(64)
    fd, dirs = _fd_cells_and_directions(phi, 2000, nthreads, cells, 2, seed=640)
    return phi, cells, fd, dirs


@pytest.mark.parametrize("precision,tol", [("f64", 1e-6), ("f32", 1e-3)])
def test_adjoint_at_64_squared_matches_oracle_central_differences(fd_64, precision, tol):
    import torch

    from paper_1308_2071_gb300 import Cavity

    phi, cells, fd, dirs = fd_64
    cav = Cavity(64, 64, Ra=1e5, Da=1e-2, phi=0.6, precision=precision, phi_field=torch.from_numpy(phi).cuda())
    _, g = cav.adjoint(2000, 100)
    g = g.double().cpu().numpy()
    ad = np.array([g[y, x] for (x, y) in cells] + [float((g * v).sum()) for v in dirs])
    err = np.linalg.norm(ad - fd) / np.linalg.norm(fd)
    assert err < tol, (precision, err, list(zip(ad, fd)))
    cav.close()


def test_adjoint_at_512_squared_along_random_directions(nthreads):
    # The gradient benchmark itself: 512^2, 2000 steps, checkpoint every 100,
    # FP32 storage; its gradient along two random unit directions against
    # central differences of the FP64 oracle (four oracle runs of 5.2e8 node
    # updates each).
    import torch

    from paper_1308_2071_gb300 import Cavity
    from paper_1308_2071_gb300.inputs import perturbed_porosity

    n = 512
    phi = perturbed_porosity(n, n, phi_bar=0.6, amplitude=0.05, corr_len=8.0, seed=2000)
    fd, dirs = _fd_cells_and_directions(phi, 2000, nthreads, [], 2, seed=512)
    cav = Cavity(n, n, Ra=1e5, Da=1e-2, phi=0.6, precision="f32", phi_field=torch.from_numpy(phi).cuda())
    _, g = cav.adjoint(2000, 100)
    g = g.double().cpu().numpy()
    ad = np.array([float((g * v).sum()) for v in dirs])
    err = np.linalg.norm(ad - fd) / np.linalg.norm(fd)
    assert err < 1e-3, (err, list(zip(ad, fd)))
    cav.close()
