"""mm_step_host: steps from a host-resident state with the result written
back to host memory must equal mm_set_m + mm_step + mm_get_m bit for bit,
whether the kernels reach the host buffers directly (page-locked, or
pageable on a device with coherent host access) or the data is staged."""
import numpy as np
import pytest

from paper_1406_7459_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MS, A_EX, GAMMA = 8.6e5, 1.3e-11, inputs.GAMMA0


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _ctx(grid):
    from paper_1406_7459_gb300 import mm
    ctx = mm.mm_create(grid, (4e-9, 4e-9, 4e-9), MS, A_EX, 5e2, 0.05, GAMMA)
    mm.mm_set_field(ctx, (-2.46e4, 4.34e3, 0.0))
    return ctx


def _reference(grid, M, n, dt):
    from paper_1406_7459_gb300 import mm
    ctx = _ctx(grid)
    mm.mm_set_m(ctx, torch.from_numpy(M).cuda())
    mm.mm_step(ctx, n, dt)
    out = torch.empty(3 * ctx.N, device="cuda")
    mm.mm_get_m(ctx, out)
    mm.mm_sync(ctx)
    return out.cpu().numpy()


# the fused film path (256x256x4, 64x64x4), the generic and the thick paths
@pytest.mark.parametrize("grid", [(256, 256, 4), (64, 64, 4), (20, 12, 3), (32, 32, 16)])
@pytest.mark.parametrize("pinned", [True, False])
def test_step_host_equals_set_step_get(grid, pinned):
    from paper_1406_7459_gb300 import mm
    M = np.ascontiguousarray(inputs.perturbed_m(grid, MS, seed=41, amplitude=0.3).reshape(-1), np.float32)
    ref1 = _reference(grid, M, 1, 5e-14)
    ref3 = _reference(grid, M, 3, 5e-14)
    ctx = _ctx(grid)
    if pinned:
        Min = torch.from_numpy(M.copy()).pin_memory()
        Mout = torch.empty_like(Min).pin_memory()
    else:
        Min = M.copy()
        Mout = np.empty_like(M)
    mm.mm_step_host(ctx, Min, 1, 5e-14, Mout)
    got = Mout.numpy() if pinned else Mout
    assert np.array_equal(got, ref1)
    # again from the caller's buffer, three steps, in place in the output
    Mio = torch.from_numpy(M.copy()).pin_memory() if pinned else M.copy()
    mm.mm_step_host(ctx, Mio, 3, 5e-14, Mio)
    got3 = Mio.numpy() if pinned else Mio
    assert np.array_equal(got3, ref3)
    # the context's state is the result
    dev = torch.empty(3 * ctx.N, device="cuda")
    mm.mm_get_m(ctx, dev)
    mm.mm_sync(ctx)
    assert np.array_equal(dev.cpu().numpy(), ref3)
