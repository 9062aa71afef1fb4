"""Batched sweep (one persistent, graph-captured launch for many cavities):
bitwise agreement with the single-cavity kernel, FP64 parity with the oracle,
the bounded grid barrier's timeout status, and the autotuner's cache."""
import numpy as np
import pytest

from oracle import Oracle, derive

pytestmark = pytest.mark.gpu

CAVS = [dict(nx=37, ny=41, Ra=1e5, Da=1e-2, phi=0.6),
        dict(nx=64, ny=64, Ra=1e4, Da=1e-1, phi=0.3),
        dict(nx=100, ny=80, Ra=1e6, Da=1e-4, phi=0.9),
        dict(nx=129, ny=131, Ra=3e5, Da=3e-3, phi=0.45),
        dict(nx=5, ny=7, Ra=1e3, Da=1e-2, phi=0.5)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def np_(t):
    return t.double().cpu().numpy()


def test_batch_matches_single_cavity_bit_for_bit():
    from paper_1308_2071_gb300 import Batch, Cavity

    b = Batch(CAVS, precision="f32")
    b.step(1)
    b.step(299)  # two captured graphs of different length
    hot, cold = b.nusselt()
    rc, st = b.status()
    assert rc == 0 and not st.any()
    assert b.query()["t"] == 300
    for k, cv in enumerate(CAVS):
        c = Cavity(cv["nx"], cv["ny"], Ra=cv["Ra"], Da=cv["Da"], phi=cv["phi"], precision="f32",
                   nodes_per_thread=1)  # the batched kernel runs the one-node code path
        c.step(300)
        f1, g1 = c.read_state()
        f2, g2 = b.read_state(k)
        assert np.array_equal(np_(f1), np_(f2)), k
        assert np.array_equal(np_(g1), np_(g2)), k
        nh, nc = c.nusselt()  # same temperatures, reduction summed in another order
        assert abs(nh - hot[k]) <= 1e-12 * abs(nh) and abs(nc - cold[k]) <= 1e-12 * abs(nc), k
        c.close()
    b.close()


# (tile_w, tile_h, blocks_per_sm, scheduling); tile_h = 0: runs of tile_w consecutive nodes, -1: runs of
# tile_w node pairs, -2: node pairs over each cavity's interior and its border in tiles of their own
@pytest.mark.parametrize("tiles", [None, (64, 8, 0, 0), (32, 8, 0, 1), (128, 4, 2, 1), (32, 1, 0, 0),
                                   (32, 2, 0, 1), (64, 1, 0, 0), (32, 1, 0, 2), (32, 2, 0, 2), (128, 4, 0, 2),
                                   (32, 0, 0, 0), (64, 0, 0, 1), (256, 0, 2, 0), (512, 0, 0, 2),
                                   (64, -1, 0, 1), (32, -2, 0, 2), (128, -2, 0, 0)])
def test_batch_fp64_matches_oracle(nthreads, tiles):
    from paper_1308_2071_gb300 import Batch

    cavs = CAVS[:3]
    b = Batch(cavs, precision="f64")
    if tiles:
        b.set_tiles(*tiles)  # 512-node tiles: two nodes per thread
    b.step(250)
    hot, _ = b.nusselt()
    for k, cv in enumerate(cavs):
        o = Oracle(derive(cv["nx"], cv["ny"], Ra=cv["Ra"], Da=cv["Da"], phi=cv["phi"])).step(250, threads=nthreads)
        fo, go = o.state()
        f, g = b.read_state(k)
        assert np.abs(np_(f) - fo).max() < 1e-12, k
        assert np.abs(np_(g) - go).max() < 1e-12, k
        assert abs(hot[k] - o.nusselt()[0]) < 1e-10 * abs(hot[k]), k
    b.close()


@pytest.mark.parametrize("tiles,precision", [((32, 1, 0, 2), "f32"), ((32, 0, 0, 2), "f32"),
                                             ((32, 0, 0, 0), "f32"), ((256, 0, 0, 1), "f32"),
                                             ((32, 1, 0, 2), "f32t"), ((256, 1, 0, 0), "f32t")])
def test_one_node_tiles_are_bit_identical_to_the_single_cavity_kernel(tiles, precision):
    # one node per thread under every scheduling, rectangular or row-run
    # tiles (the 5 x 7 cavity makes a 32-node run wrap over several rows),
    # plain and framed FP32 storage
    from paper_1308_2071_gb300 import Batch, Cavity

    b = Batch(CAVS, precision=precision)
    b.set_tiles(*tiles)
    b.step(137)
    b.step(163)
    rc, st = b.status()
    assert rc == 0
    for k, cv in enumerate(CAVS):
        c = Cavity(cv["nx"], cv["ny"], Ra=cv["Ra"], Da=cv["Da"], phi=cv["phi"], precision=precision,
                   nodes_per_thread=1)
        c.step(300)
        assert np.array_equal(np_(c.read_state()[0]), np_(b.read_state(k)[0])), k
        assert np.array_equal(np_(c.read_state()[1]), np_(b.read_state(k)[1])), k
        c.close()
    b.close()


@pytest.mark.parametrize("tiles,precision", [((32, -1, 0, 1), "f32"), ((128, -1, 0, 2), "f32"),
                                             ((32, -2, 0, 0), "f32"), ((64, -2, 0, 1), "f32"),
                                             ((256, -2, 0, 2), "f32"), ((128, -2, 0, 1), "f32t")])
def test_pair_tiles_are_bit_identical_to_the_single_cavity_pair_kernel(tiles, precision):
    # runs of node pairs side by side along x (tile_h = -1), and the same over
    # each cavity's interior with the border nodes in tiles of their own
    # (tile_h = -2): every node runs the code of the single-cavity kernel in
    # launch mode 3 (the pair code clear of the walls, the one-node code on
    # and beside them), so the lattices are the same bit for bit, on even and
    # odd widths and on a 5 x 7 cavity whose runs wrap over several rows
    from paper_1308_2071_gb300 import Batch, Cavity

    b = Batch(CAVS, precision=precision)
    b.set_tiles(*tiles)
    b.step(137)
    b.step(163)
    rc, st = b.status()
    assert rc == 0
    for k, cv in enumerate(CAVS):
        c = Cavity(cv["nx"], cv["ny"], Ra=cv["Ra"], Da=cv["Da"], phi=cv["phi"], precision=precision,
                   nodes_per_thread=3, block_x=32, block_y=4)
        c.step(300)
        assert np.array_equal(np_(c.read_state()[0]), np_(b.read_state(k)[0])), k
        assert np.array_equal(np_(c.read_state()[1]), np_(b.read_state(k)[1])), k
        c.close()
    b.close()


@pytest.mark.parametrize("precision", ["f32", "f32t"])
def test_cavities_with_their_own_wall_temperatures_are_bit_identical(precision):
    # wall temperatures that differ between cavities change coefficients that
    # are otherwise batch-wide: the batch then takes every coefficient from
    # the cavity's descriptor (the other kernel variant), with the same results
    from paper_1308_2071_gb300 import Batch, Cavity

    cavs = [dict(cv) for cv in CAVS]
    cavs[1].update(Th=1.5, Tc=-0.25)
    cavs[3].update(Th=0.75)
    b = Batch([dict(cv) for cv in cavs], precision=precision)
    b.set_tiles(32, 1, 0, 1)
    b.step(200)
    for k, cv in enumerate(cavs):
        extra = {key: cv[key] for key in ("Th", "Tc") if key in cv}
        c = Cavity(cv["nx"], cv["ny"], Ra=cv["Ra"], Da=cv["Da"], phi=cv["phi"], precision=precision,
                   nodes_per_thread=1, **extra)
        c.step(200)
        assert np.array_equal(np_(c.read_state()[0]), np_(b.read_state(k)[0])), k
        assert np.array_equal(np_(c.read_state()[1]), np_(b.read_state(k)[1])), k
        c.close()
    b.close()


@pytest.mark.parametrize("tiles", [(32, 16), (64, 0), (512, 0)])
def test_two_node_tiles_agree_with_the_single_cavity_kernel(tiles):
    from paper_1308_2071_gb300 import Batch, Cavity

    b = Batch(CAVS, precision="f32")
    b.set_tiles(*tiles)
    b.step(300)
    for k, cv in enumerate(CAVS):
        c = Cavity(cv["nx"], cv["ny"], Ra=cv["Ra"], Da=cv["Da"], phi=cv["phi"], precision="f32",
                   nodes_per_thread=2)
        c.step(300)
        # same formulas; fused multiply-adds may differ: FP32 roundings over 300 steps
        assert np.abs(np_(c.read_state()[0]) - np_(b.read_state(k)[0])).max() < 2e-6, k
        c.close()
    b.close()


def test_grid_barrier_timeout_is_reported_and_context_survives():
    from paper_1308_2071_gb300 import Batch, Cavity, _lib

    b = Batch(CAVS[:4], precision="f32")
    assert b.query()["nblocks"] > 1
    b.set_wait_limit(0)  # any block that has to wait gives up at once
    b.step(8)
    rc, _ = b.status()
    assert rc == _lib.LBM_ERR_TIMEOUT
    b.set_wait_limit(20_000_000)  # clears the flag; the state is incomplete but the context is fine
    b.close()
    c = Cavity(40, 40, Ra=1e5, Da=1e-2, phi=0.6, precision="f32")
    c.step(10)
    assert c.query()[1] == 0
    c.close()


def test_autotuner_picks_a_shape_and_caches_it(tmp_path):
    from paper_1308_2071_gb300 import Batch

    cache = str(tmp_path / "tune.txt")
    b = Batch(CAVS[:4], precision="f32")
    shape = b.tune(cache)
    assert b.query()["t"] == 0  # tuning resets the lattices
    nodes = shape[0] if shape[1] == 0 else shape[0] * shape[1]  # tile_h = 0: a run of tile_w nodes
    assert nodes in (32, 64, 256, 512)
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and lines[0].split()[1:3] == [str(shape[0]), str(shape[1])]
    b.step(50)
    b2 = Batch(CAVS[:4], precision="f32")
    assert b2.tune(cache) == shape  # served from the cache
    assert len(open(cache).read().splitlines()) == 1
    b2.step(50)
    for k in range(4):
        assert np.array_equal(np_(b.read_state(k)[0]), np_(b2.read_state(k)[0]))
    b.close()
    b2.close()


def test_batch_rejects_invalid_cavity_with_its_index():
    from paper_1308_2071_gb300 import Batch, _lib

    bad = CAVS[:2] + [dict(nx=40, ny=40, Ra=1e5, Da=1e-2, phi=1.5)]
    with pytest.raises(_lib.LbmError, match="cavity 2"):
        Batch(bad, precision="f32")
