"""The allocation-free demag entry point (mm_demag_field_noalloc) must give
the same field as mm_demag_field.  It serves callers that may not allocate
device memory; its workspace is a fixed array inside the library, so two
calls in a row must not leak state into each other.  Collected last so that
a run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

from paper_1406_7459_gb300 import inputs
from tests._helpers import rel_l2, rel_max

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MS = 8.6e5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


@pytest.mark.parametrize("grid,cell", [((256, 256, 4), (4e-9, 4e-9, 4e-9)),
                                       ((48, 40, 3), (5e-9, 4e-9, 3e-9)),
                                       # thick: the split y/z pass with row stride Ly
                                       ((32, 32, 16), (4e-9, 4e-9, 4e-9))])
def test_noalloc_matches_mm_demag_field_on_two_calls(grid, cell):
    from paper_1406_7459_gb300 import mm
    ctx = mm.mm_create(grid, cell, MS, 1.3e-11, 0.0, 0.5, inputs.GAMMA0)
    (Lx, Ly, Lz), _ = mm.mm_plan_info(ctx)
    Kt = torch.empty((Lx // 2 + 1) * (Lz // 2 + 1) * (Ly // 2 + 1) * 6, dtype=torch.float32, device="cuda")
    mm.mm_kernel_spectrum(ctx, Kt)
    for seed in (11, 12):                       # two calls in a row
        M = torch.from_numpy(inputs.random_unit_m(grid, MS, seed).reshape(-1)).cuda()
        H_ref = torch.empty_like(M)
        mm.mm_demag_field(ctx, M, H_ref)
        H = torch.full_like(M, float("nan"))
        mm.mm_demag_field_noalloc(grid, Kt, M, H)
        torch.cuda.synchronize()
        a, b = H.cpu().numpy().astype(np.float64), H_ref.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(a))
        assert rel_l2(a, b) < 1e-5
        assert rel_max(a, b) < 1e-5


def test_noalloc_rejects_a_spectrum_of_the_wrong_size():
    from paper_1406_7459_gb300 import mm
    grid, cell = (48, 40, 3), (5e-9, 4e-9, 3e-9)
    ctx = mm.mm_create(grid, cell, MS, 1.3e-11, 0.0, 0.5, inputs.GAMMA0)
    (Lx, Ly, Lz), _ = mm.mm_plan_info(ctx)
    n_kt = (Lx // 2 + 1) * (Lz // 2 + 1) * (Ly // 2 + 1) * 6
    Kt = torch.zeros(n_kt - 6, dtype=torch.float32, device="cuda")   # a smaller grid's size
    M = torch.zeros(3 * 48 * 40 * 3, device="cuda")
    H = torch.zeros_like(M)
    with pytest.raises(mm.MMError) as e:
        mm.mm_demag_field_noalloc(grid, Kt, M, H)
    assert e.value.code == mm.MM_EINVAL
    assert "Kt" in str(e.value)


def test_noalloc_rejects_grids_beyond_its_workspace():
    from paper_1406_7459_gb300 import mm
    grid = (512, 512, 8)
    n = 3 * 512 * 512 * 8
    M = torch.zeros(n, device="cuda")
    H = torch.zeros(n, device="cuda")
    Kt = torch.zeros(8, device="cuda")
    with pytest.raises(mm.MMError) as e:
        mm.mm_demag_field_noalloc(grid, Kt, M, H)
    assert e.value.code == mm.MM_EUNSUPPORTED
    assert "workspace" in str(e.value)
