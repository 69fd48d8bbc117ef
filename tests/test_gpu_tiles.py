"""Tile shapes of the sweep kernels (elements per reconstruction block,
predictor block size, blocks per SM) change no result: every shape gives the
same state bit for bit.  The autotuner times them on the loaded state, keeps
the fastest and leaves the state as it was."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1408_3719_gb300 import workloads as W  # noqa: E402

SHAPES = [(rh, pw, bp) for rh in (0, 1) for pw in (0, 1) for bp in (4, 8, 16)]
KEYS = ("Q", "QM", "X", "t", "dt", "count", "qhat")


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_3719_gb300 import aleweno
    return aleweno


@pytest.mark.parametrize("order", [1, 2, 3])
def test_every_tile_shape_gives_the_same_state(order):
    aleweno = _need_gpu()
    mesh, Q = W.explosion(0.02)
    s = aleweno.Solver(order_M=order, t_end=0.25)
    s.load_mesh(mesh)
    ref = None
    for shape in SHAPES:
        s.set_tiles(*shape)
        s.load_state(Q)
        s.enqueue(60)
        s.sync()
        e = s.get_elem()
        nX, nt = s.get_nodes()
        if ref is None:
            ref = (e, nX, nt)
            assert e["count"].sum() > 100
            continue
        for k in KEYS:
            assert np.array_equal(e[k], ref[0][k]), (shape, k)
        assert np.array_equal(nX, ref[1]) and np.array_equal(nt, ref[2]), shape


def test_autotune_keeps_the_state_and_picks_a_shape():
    aleweno = _need_gpu()
    mesh, Q = W.explosion(0.02)
    s = aleweno.Solver(order_M=2, t_end=0.25)
    s.load_mesh(mesh)
    s.load_state(Q)
    s.enqueue(5)
    s.sync()
    before = s.get_elem()
    best, table = s.autotune(4)
    after = s.get_elem()
    for k in KEYS:
        assert np.array_equal(before[k], after[k]), k
    assert (best["recon_half"], best["pred_wide"], best["bpsm"]) in table
    assert all(v > 0 for v in table.values())
    assert s.get_tiles() == best
    # the run continues from the kept state with the chosen shape exactly as
    # with the default shape
    s.enqueue(6)
    s.sync()
    tuned = s.get_elem()
    s.set_tiles(0, 0, 8)
    s.load_state(Q)
    s.enqueue(11)
    s.sync()
    plain = s.get_elem()
    for k in KEYS:
        assert np.array_equal(tuned[k], plain[k]), k
