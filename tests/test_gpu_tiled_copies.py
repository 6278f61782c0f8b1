"""The x-step kernel's tiled tensor copies (mm_set_tiled_copies): the gather
of the plane kernel's output and the scatter of the next spectrum as one
4-D box per block instead of per-thread 16-byte copies and stores.

The arithmetic between the copies is the same, so every mask must give the
default path's bits: Euler steps (direct programmatic launch chains for
single steps, the 16-step graph), the field evaluations that end in the x-step
kernel (H_demag, H_eff) and steps of a host-resident state.  The default
path is pinned to the FP64 oracle by the parity tests.
"""
import numpy as np
import pytest

from paper_1406_7459_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MS, A_EX, GAMMA = 8.6e5, 1.3e-11, inputs.GAMMA0
CELL = (4e-9, 4e-9, 4e-9)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1406_7459_gb300 import mm
    mm.lib()


def _mm():
    from paper_1406_7459_gb300 import mm
    return mm


def _ctx(grid, mask):
    mm = _mm()
    ctx = mm.mm_create(grid, CELL, MS, A_EX, 5e2, 0.02, GAMMA)
    mm.mm_set_tiled_copies(ctx, mask)
    assert mm.mm_get_tiled_copies(ctx) == mask
    mm.mm_set_field(ctx, (-2.46e4, 4.34e3, 1.0e3))
    return ctx


def _steps(grid, M, mask, runs=(1, 3, 20), dt=5e-14):
    mm = _mm()
    ctx = _ctx(grid, mask)
    mm.mm_set_m(ctx, torch.from_numpy(M.reshape(-1)).cuda())
    for n in runs:
        mm.mm_step(ctx, n, dt)
    out = torch.empty(3 * ctx.N, device="cuda")
    mm.mm_get_m(ctx, out)
    mm.mm_sync(ctx)
    return out.cpu().numpy()


GRIDS = [(256, 256, 4), (128, 128, 2), (64, 64, 4), (32, 32, 1)]


@pytest.mark.parametrize("grid", GRIDS)
def test_tiled_copies_step_bitwise(grid):
    mm = _mm()
    M = np.ascontiguousarray(inputs.perturbed_m(grid, MS, seed=41, amplitude=0.3), np.float32)
    ref = _steps(grid, M, 0)
    assert np.all(np.isfinite(ref))
    for mask in (mm.MM_TILED_GATHER, mm.MM_TILED_SCATTER, mm.MM_TILED_GATHER | mm.MM_TILED_SCATTER):
        assert np.array_equal(_steps(grid, M, mask), ref), mask


@pytest.mark.parametrize("grid", [(256, 256, 4), (64, 64, 2)])
def test_tiled_copies_fields_bitwise(grid):
    mm = _mm()
    M = torch.from_numpy(np.ascontiguousarray(inputs.random_unit_m(grid, MS, seed=42), np.float32).reshape(-1)).cuda()
    out = {}
    for mask in (0, mm.MM_TILED_GATHER | mm.MM_TILED_SCATTER):
        ctx = _ctx(grid, mask)
        hd, he = torch.empty_like(M), torch.empty_like(M)
        mm.mm_demag_field(ctx, M, hd)
        mm.mm_effective_field(ctx, M, he)
        mm.mm_sync(ctx)
        out[mask] = (hd.cpu().numpy(), he.cpu().numpy())
    assert np.any(out[0][0] != 0)
    assert np.array_equal(out[0][0], out[3][0])
    assert np.array_equal(out[0][1], out[3][1])


def test_tiled_copies_host_steps_and_switching():
    """mm_step_host with tiled copies equals the default; switching the mask
    on a live context re-captures the step graphs (same bits either way)."""
    mm = _mm()
    grid = (256, 256, 4)
    M = np.ascontiguousarray(inputs.perturbed_m(grid, MS, seed=43, amplitude=0.3), np.float32).reshape(-1)
    ref = _steps(grid, M, 0, runs=(5,))
    ctx = _ctx(grid, mm.MM_TILED_GATHER | mm.MM_TILED_SCATTER)
    Mh = torch.from_numpy(M.copy()).pin_memory()
    Mo = torch.empty_like(Mh).pin_memory()
    mm.mm_step_host(ctx, Mh, 5, 5e-14, Mo)
    assert np.array_equal(Mo.numpy(), ref)
    # 16-step graph captured with one mask, replayed after switching
    ctx = _ctx(grid, 0)
    mm.mm_set_m(ctx, torch.from_numpy(M).cuda())
    mm.mm_step(ctx, 16, 5e-14)
    mm.mm_set_tiled_copies(ctx, mm.MM_TILED_GATHER | mm.MM_TILED_SCATTER)
    mm.mm_step(ctx, 16, 5e-14)
    a = torch.empty(3 * ctx.N, device="cuda")
    mm.mm_get_m(ctx, a)
    mm.mm_sync(ctx)
    assert np.array_equal(a.cpu().numpy(), _steps(grid, M, 0, runs=(16, 16)))


def test_tiled_copies_setter_errors():
    mm = _mm()
    ctx = mm.mm_create((256, 256, 4), CELL, MS, A_EX, 0.0, 0.5, GAMMA)
    assert mm.mm_get_tiled_copies(ctx) == 0
    with pytest.raises(mm.MMError) as e:
        mm.mm_set_tiled_copies(ctx, 4)
    assert e.value.code == mm.MM_EINVAL
    # no tiled form: the generic mixed-radix path, and an x extent whose box
    # would be longer than a tensor map allows
    for grid in ((200, 60, 3), (512, 512, 1)):
        ctx = mm.mm_create(grid, CELL, MS, A_EX, 0.0, 0.5, GAMMA)
        mm.mm_set_tiled_copies(ctx, 0)
        with pytest.raises(mm.MMError) as e:
            mm.mm_set_tiled_copies(ctx, mm.MM_TILED_GATHER)
        assert e.value.code == mm.MM_EUNSUPPORTED
        assert mm.mm_get_tiled_copies(ctx) == 0
