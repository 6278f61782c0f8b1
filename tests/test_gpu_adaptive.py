"""GPU parity of the adaptive Dormand-Prince run (mm_run_adaptive) against
the FP64 oracle's run_dopri5 on the same seeded FP32 start.

The controller decisions depend on the FP32 error estimate, which carries
rounding of order 1e-7 |dt k| against an estimate of order tol, so the GPU
and the oracle may take slightly different step sequences; the checks
compare what that leaves unique: the state after one fixed trial step, the
error estimate behind the proposed next step, and final states that agree
to a small multiple of the accumulated tolerance.
"""
import numpy as np
import pytest

from oracle import llg as L
from paper_1406_7459_gb300 import inputs
from tests._helpers import oracle_spectrum, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MS, A_EX, GAMMA = 8.6e5, 1.3e-11, inputs.GAMMA0
KU, ALPHA, HEXT = 1e4, 0.2, (2e4, -1e4, 5e3)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1406_7459_gb300 import mm
    mm.lib()


def _mm():
    from paper_1406_7459_gb300 import mm
    return mm


def _setup(grid, cell, seed):
    M = inputs.perturbed_m(grid, MS, seed=seed, amplitude=0.3)
    ctx = _mm().mm_create(grid, cell, MS, A_EX, KU, ALPHA, GAMMA)
    _mm().mm_set_field(ctx, HEXT)
    _mm().mm_set_m(ctx, torch.from_numpy(np.ascontiguousarray(M, np.float32).reshape(-1)).cuda())
    return ctx, M


def _state(ctx, grid):
    out = torch.empty(3 * ctx.N, device="cuda")
    _mm().mm_get_m(ctx, out)
    _mm().mm_sync(ctx)
    nx, ny, nz = grid
    return out.cpu().numpy().reshape(3, nz, ny, nx).astype(np.float64)


GRIDS = [((16, 16, 2), (4e-9, 4e-9, 3e-9)), ((20, 12, 3), (5e-9, 5e-9, 3e-9))]


@pytest.mark.parametrize("grid,cell", GRIDS)
def test_one_dormand_prince_step_and_its_error_estimate(grid, cell):
    """t_span = dt with a loose tol: one accepted step.  The state matches
    the oracle's step; the error estimate, recovered from the proposed next
    step h * 0.9 (tol/err)^(1/5) (unclamped by the choice of tol), matches
    the oracle's to 2 %."""
    ctx, M = _setup(grid, cell, seed=71)
    Kt, Lp = oracle_spectrum(grid, cell)
    args = (cell, MS, A_EX, KU, ALPHA, GAMMA, HEXT, Kt, Lp)
    M64 = M.astype(np.float64)
    dt = 2e-13
    ref, err_ref, _ = L.dopri5_step(M64, L._rhs(M64, *args), dt, *args)
    tol = err_ref * 2.0                      # accepted, factor 0.9 * 2^(1/5) inside the clamp
    done, dt_next, st = _mm().mm_run_adaptive(ctx, dt, dt, tol, 10)
    assert done and st["accepted"] == 1 and st["rejected"] == 0 and st["evaluations"] == 7
    got = _state(ctx, grid)
    assert rel_l2(got - M64, ref - M64) < 1e-4
    assert rel_l2(got, ref) < 1e-6
    err_gpu = tol * (0.9 * dt / dt_next) ** 5
    assert abs(err_gpu / err_ref - 1.0) < 2e-2, (err_gpu, err_ref)


@pytest.mark.parametrize("grid,cell", GRIDS)
def test_adaptive_run_matches_oracle(grid, cell):
    """A run of a few tens of steps from a deliberately large first trial step
    (so that the controller rejects and shrinks first): step counts within
    10 % and final states within a small multiple of the accumulated tol."""
    ctx, M = _setup(grid, cell, seed=72)
    Kt, Lp = oracle_spectrum(grid, cell)
    t_span, dt0, tol = 2e-11, 5e-12, 1e-6
    ref, dt_ref, (acc, rej, nev, t) = L.run_dopri5(M.astype(np.float64), t_span, dt0, tol, 10000, cell, MS, A_EX,
                                                   KU, ALPHA, GAMMA, HEXT, Kt, Lp)
    done, dt_next, st = _mm().mm_run_adaptive(ctx, t_span, dt0, tol, 10000)
    assert done and abs(st["t"] - t_span) < 1e-12 * t_span
    assert rej >= 1 and st["rejected"] >= 1
    assert abs(st["accepted"] - acc) <= max(1, acc // 10), (st, acc)
    assert st["evaluations"] == 1 + 6 * (st["accepted"] + st["rejected"])
    got = _state(ctx, grid)
    M64 = M.astype(np.float64)
    assert rel_l2(got - M64, ref - M64) < 20 * tol * acc
    norms = np.sqrt(np.sum(got * got, axis=0))
    assert np.max(np.abs(norms - MS)) < 1e-6 * MS


def test_adaptive_run_step_limit_and_arguments():
    """A run stopped by its step limit.  The first trial step is small enough
    that the first two error estimates lie far below tol (0.9 (tol/err)^(1/5)
    > 5, so the controller's growth clamps at 5 on both sides whatever the
    FP32 rounding of the estimate): the GPU and the oracle take the same
    steps dt0, 5 dt0, 25 dt0, all accepted, and the states compare
    directly, as after one step."""
    grid, cell = GRIDS[0]
    ctx, M = _setup(grid, cell, seed=73)
    Kt, Lp = oracle_spectrum(grid, cell)
    t_span, dt0, tol = 2e-11, 4e-15, 1e-4
    ref, dt_ref, (acc, rej, nev, t) = L.run_dopri5(M.astype(np.float64), t_span, dt0, tol, 3, cell, MS, A_EX, KU,
                                                   ALPHA, GAMMA, HEXT, Kt, Lp)
    assert (acc, rej) == (3, 0) and abs(t - 31 * dt0) < 1e-9 * t
    done, dt_next, st = _mm().mm_run_adaptive(ctx, t_span, dt0, tol, 3)
    assert not done and st["accepted"] == 3 and st["rejected"] == 0 and st["evaluations"] == 19
    assert abs(st["t"] - t) < 1e-9 * t
    got = _state(ctx, grid)
    M64 = M.astype(np.float64)
    assert rel_l2(got, ref) < 1e-6
    assert rel_l2(got - M64, ref - M64) < 1e-4
    # the proposed next step follows the third (unclamped) error estimate
    assert abs(dt_next / dt_ref - 1.0) < 2e-2, (dt_next, dt_ref)
    mm = _mm()
    for bad in ((t_span, -1.0, tol, 10), (t_span, dt0, 0.0, 10), (t_span, dt0, tol, 0), (-1.0, dt0, tol, 10)):
        with pytest.raises(mm.MMError) as ei:
            mm.mm_run_adaptive(ctx, *bad)
        assert ei.value.code == mm.MM_EINVAL
    # t_span = 0 leaves the state alone
    before = _state(ctx, grid)
    done, _, st = mm.mm_run_adaptive(ctx, 0.0, dt0, tol, 10)
    assert done and st["accepted"] == 0 and np.array_equal(_state(ctx, grid), before)
