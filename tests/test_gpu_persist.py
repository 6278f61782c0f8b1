"""The persistent Euler step (one cooperative launch per mm_step call: plane
phase, grid barrier, x-step phase per step) against the two-kernel graph
step it replaces, and its bounded grid-barrier wait.

Both run the same arithmetic in the same order, so the states must agree
bit for bit after any number of steps; the graph path itself is pinned to
the FP64 oracle by the parity tests, and the first case here checks the
persistent run against the oracle directly as well.
"""
import numpy as np
import pytest

from oracle import llg as L
from paper_1406_7459_gb300 import inputs
from tests._helpers import oracle_spectrum, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MS, A_EX, GAMMA = 8.6e5, 1.3e-11, inputs.GAMMA0


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1406_7459_gb300 import mm
    mm.lib()


def _mm():
    from paper_1406_7459_gb300 import mm
    return mm


def _run(grid, cell, M, path, runs, dt=5e-14, Ku=5e2, alpha=0.02, Hext=(-2.46e4, 4.34e3, 0.0)):
    mm = _mm()
    ctx = mm.mm_create(grid, cell, MS, A_EX, Ku, alpha, GAMMA)
    mm.mm_set_step_path(ctx, path)
    mm.mm_set_field(ctx, Hext)
    mm.mm_set_m(ctx, torch.from_numpy(np.ascontiguousarray(M, np.float32).reshape(-1)).cuda())
    for n in runs:
        mm.mm_step(ctx, n, dt)
    out = torch.empty(3 * ctx.N, device="cuda")
    mm.mm_get_m(ctx, out)
    mm.mm_sync(ctx)
    return ctx, out.cpu().numpy()


PERSIST_GRIDS = [(256, 256, 4), (128, 128, 4), (64, 64, 4), (256, 256, 2), (256, 256, 1)]


@pytest.mark.parametrize("grid", PERSIST_GRIDS)
def test_persistent_step_is_bitwise_the_graph_step(grid):
    """Runs of 1, 3 and 20 steps (the graph path takes direct programmatic
    launch chains for single steps and a 16-step graph; the persistent path
    one launch per call) from a random start: equal bits."""
    mm = _mm()
    cell = (4e-9, 4e-9, 4e-9)
    M = inputs.perturbed_m(grid, MS, seed=31, amplitude=0.3)
    runs = (1, 3, 20)
    cp, a = _run(grid, cell, M, mm.MM_STEP_PERSISTENT, runs)
    cg, b = _run(grid, cell, M, mm.MM_STEP_GRAPH, runs)
    assert mm.mm_get_step_path(cp) == mm.MM_STEP_PERSISTENT
    assert mm.mm_get_step_path(cg) == mm.MM_STEP_GRAPH
    assert np.all(np.isfinite(a))
    assert np.array_equal(a, b)


def test_persistent_step_matches_the_oracle():
    """Seven persistent steps of the 64x64x4 film against the FP64 oracle's
    Euler run (the tolerance of the other step tests)."""
    mm = _mm()
    grid, cell = (64, 64, 4), (4e-9, 4e-9, 4e-9)
    M = inputs.random_unit_m(grid, MS, seed=32)
    Ku, alpha, dt, Hext = 2e4, 0.3, 1e-13, (5e3, 1e4, -2e3)
    ctx, got = _run(grid, cell, M, mm.MM_STEP_PERSISTENT, (7,), dt=dt, Ku=Ku, alpha=alpha, Hext=Hext)
    Kt, Lp = oracle_spectrum(grid, cell)
    ref = L.run_euler(M.astype(np.float64), 7, dt, cell, MS, A_EX, Ku, alpha, GAMMA, Hext, Kt, Lp)
    got = got.reshape(ref.shape).astype(np.float64)
    assert rel_l2(got, ref) < 1e-5
    assert np.max(np.abs(np.sqrt(np.sum(got * got, axis=0)) - MS)) < 1e-6 * MS


def test_auto_path_and_grids_without_a_persistent_step():
    mm = _mm()
    ctx = mm.mm_create((256, 256, 4), (4e-9,) * 3, MS, A_EX, 0.0, 0.5, GAMMA)
    assert mm.mm_get_step_path(ctx) == mm.MM_STEP_GRAPH               # the default (faster here)
    mm.mm_set_step_path(ctx, mm.MM_STEP_PERSISTENT)
    assert mm.mm_get_step_path(ctx) == mm.MM_STEP_PERSISTENT
    mm.mm_set_step_path(ctx, mm.MM_STEP_AUTO)
    assert mm.mm_get_step_path(ctx) == mm.MM_STEP_GRAPH
    for grid in ((200, 60, 3), (32, 16, 2), (64, 64, 16)):
        ctx = mm.mm_create(grid, (4e-9,) * 3, MS, A_EX, 0.0, 0.5, GAMMA)
        assert mm.mm_get_step_path(ctx) == mm.MM_STEP_GRAPH
        with pytest.raises(mm.MMError) as e:
            mm.mm_set_step_path(ctx, mm.MM_STEP_PERSISTENT)
        assert e.value.code == mm.MM_EUNSUPPORTED
    with pytest.raises(mm.MMError) as e:
        mm.mm_set_step_path(ctx, 7)
    assert e.value.code == mm.MM_EINVAL
    with pytest.raises(mm.MMError) as e:
        mm.mm_set_wait_limit(ctx, -1)
    assert e.value.code == mm.MM_EINVAL


def test_grid_barrier_wait_gives_up_and_the_context_recovers():
    """A poll limit of 0 makes every grid-barrier wait give up at once: the
    blocks leave, mm_sync reports MM_ETIMEOUT.  No GPU fault is involved.
    With the limit restored and the state set again, the next run equals the
    graph path bit for bit (the barrier counters were left clean)."""
    mm = _mm()
    grid, cell = (256, 256, 4), (4e-9, 4e-9, 4e-9)
    M = inputs.perturbed_m(grid, MS, seed=33, amplitude=0.3)
    Md = torch.from_numpy(np.ascontiguousarray(M, np.float32).reshape(-1)).cuda()
    ctx = mm.mm_create(grid, cell, MS, A_EX, 5e2, 0.02, GAMMA)
    mm.mm_set_step_path(ctx, mm.MM_STEP_PERSISTENT)
    mm.mm_set_m(ctx, Md)
    mm.mm_set_wait_limit(ctx, 0)
    mm.mm_step(ctx, 3, 5e-14)
    with pytest.raises(mm.MMError) as e:
        mm.mm_sync(ctx)
    assert e.value.code == mm.MM_ETIMEOUT
    mm.mm_set_wait_limit(ctx, 1 << 20)
    mm.mm_set_m(ctx, Md)
    mm.mm_step(ctx, 5, 5e-14)
    a = torch.empty_like(Md)
    mm.mm_get_m(ctx, a)
    mm.mm_sync(ctx)
    _, b = _run(grid, cell, M, mm.MM_STEP_GRAPH, (5,), Hext=(0.0, 0.0, 0.0))
    assert np.array_equal(a.cpu().numpy(), b)
