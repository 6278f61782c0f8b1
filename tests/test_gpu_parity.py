"""GPU parity: every step of the hot path, called through the C ABI, against
the FP64 oracle on the same seeded FP32 inputs.

Tolerances (relative L2 over the whole field, plus max-abs over the max):
H_demag <= 1e-5 per evaluation and M <= 1e-4 after the 1000-step thin-film
run; the FP64 tensor matches to 1e-10 of its largest entry; the FP32
spectrum to 1e-6; energies to 1e-6 of the largest term.
"""
import numpy as np
import pytest

from oracle import tensor as T, demag as D, llg as L
from paper_1406_7459_gb300 import inputs
from tests._helpers import padded_length, oracle_octant, oracle_spectrum, rel_l2, rel_max

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


def _ctx(grid, cell, Ms=MS, A=A_EX, Ku=0.0, alpha=0.5, gamma=GAMMA):
    return _mm().mm_create(grid, cell, Ms, A, Ku, alpha, gamma)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32).reshape(-1)).cuda()


def _host(t, grid):
    nx, ny, nz = grid
    torch.cuda.synchronize()
    return t.cpu().numpy().reshape(3, nz, ny, nx).astype(np.float64)


TENSOR_CASES = [((1, 1, 1), (3e-9, 3e-9, 3e-9)), ((5, 3, 2), (5e-9, 4e-9, 3e-9)),
                ((8, 8, 4), (5e-9, 5e-9, 3e-9)), ((32, 32, 1), (5e-9, 5e-9, 3e-9)),
                ((64, 64, 4), (4e-9, 4e-9, 4e-9)), ((40, 12, 3), (2.5e-9, 2.5e-9, 2.5e-9))]


@pytest.mark.parametrize("grid,cell", TENSOR_CASES)
def test_tensor_octant_fp64(grid, cell):
    ctx = _ctx(grid, cell)
    got = _mm().mm_tensor_octant(ctx)
    ref = oracle_octant(grid, cell)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) <= 1e-10 * scale


@pytest.mark.parametrize("grid,cell", TENSOR_CASES)
def test_kernel_spectrum_fp32(grid, cell):
    ctx = _ctx(grid, cell)
    (Lx, Ly, Lz), _ = _mm().mm_plan_info(ctx)
    assert (Lx, Ly, Lz) == tuple(padded_length(n) for n in grid)
    got = _mm().mm_kernel_spectrum(ctx)                 # [kx][kz][ky][c]
    Kt, _ = oracle_spectrum(grid, cell, (Lx, Ly, Lz))   # (6, Lz, Ly, Lx//2+1)
    ref = Kt.real[:, :Lz // 2 + 1, :Ly // 2 + 1, :].transpose(3, 1, 2, 0) / (Lx * Ly * Lz)
    assert rel_max(got, ref) < 1e-6


DEMAG_GRIDS = [(1, 1, 1), (2, 3, 1), (5, 3, 2), (7, 5, 3), (8, 8, 4), (32, 32, 1), (17, 9, 2),
               (33, 1, 1), (1, 40, 1), (3, 3, 8), (64, 64, 4), (200, 60, 3), (24, 20, 5),
               (30, 11, 6), (13, 7, 7)]


@pytest.mark.parametrize("grid", DEMAG_GRIDS)
def test_demag_field(grid):
    cell = (5e-9, 4e-9, 3e-9)
    M = inputs.random_unit_m(grid, MS, seed=sum(grid))
    ctx = _ctx(grid, cell)
    Md = _dev(M)
    Hd = torch.empty_like(Md)
    _mm().mm_demag_field(ctx, Md, Hd)
    Kt, Lp = oracle_spectrum(grid, cell)
    ref = D.demag_fft(M.astype(np.float64), Kt, Lp)
    got = _host(Hd, grid)
    assert rel_l2(got, ref) < 1e-5
    assert rel_max(got, ref) < 1e-5


@pytest.mark.parametrize("grid", [(24, 20, 4), (64, 32, 4), (32, 64, 2), (128, 16, 8), (16, 16, 1), (16, 32, 16),
                                  (16, 512, 8)])
def test_effective_field(grid):
    """H_eff of Eq. (2) against the oracle: the three-pass path (24x20x4)
    and, on power-of-two films, the plane kernel with the exchange-folded
    spectrum plus the field-only x-step kernel."""
    cell = (5e-9, 4e-9, 3e-9)
    Ku, Hext = 4e4, (1.2e4, -3e3, 2e4)
    M = inputs.random_unit_m(grid, MS, seed=9)
    ctx = _ctx(grid, cell, Ku=Ku)
    _mm().mm_set_field(ctx, Hext)
    Md = _dev(M)
    Hd = torch.empty_like(Md)
    _mm().mm_effective_field(ctx, Md, Hd)
    Kt, Lp = oracle_spectrum(grid, cell)
    M64 = M.astype(np.float64)
    ref = L.h_effective(M64, cell, MS, A_EX, Ku, Hext, D.demag_fft(M64, Kt, Lp))
    assert rel_l2(_host(Hd, grid), ref) < 1e-5


@pytest.mark.parametrize("graphs", ["1", "0"])
def test_steps_match_oracle(graphs, monkeypatch):
    monkeypatch.setenv("MM_NO_GRAPHS", "1" if graphs == "0" else "0")
    grid, cell = (20, 12, 3), (5e-9, 5e-9, 3e-9)
    Ku, alpha, dt, Hext = 2e4, 0.3, 1e-13, (5e3, 1e4, -2e3)
    M = inputs.random_unit_m(grid, MS, seed=21)
    ctx = _ctx(grid, cell, Ku=Ku, alpha=alpha)
    _mm().mm_set_field(ctx, Hext)
    _mm().mm_set_m(ctx, _dev(M))
    n = 7
    _mm().mm_step(ctx, n, dt)
    out = torch.empty(3 * ctx.N, device="cuda")
    _mm().mm_get_m(ctx, out)
    _mm().mm_sync(ctx)
    Kt, Lp = oracle_spectrum(grid, cell)
    ref = L.run_euler(M.astype(np.float64), n, dt, cell, MS, A_EX, Ku, alpha, GAMMA, Hext, Kt, Lp)
    got = _host(out, grid)
    assert rel_l2(got, ref) < 1e-5
    assert np.max(np.abs(np.sqrt(np.sum(got * got, axis=0)) - MS)) < 1e-6 * MS


def test_graph_and_direct_launches_are_bitwise_equal(monkeypatch):
    grid, cell = (16, 16, 2), (5e-9, 5e-9, 3e-9)
    M = inputs.random_unit_m(grid, MS, seed=5)
    outs = []
    for flag in ("0", "1"):
        monkeypatch.setenv("MM_NO_GRAPHS", flag)
        ctx = _ctx(grid, cell)
        _mm().mm_set_m(ctx, _dev(M))
        _mm().mm_step(ctx, 5, 1e-13)
        o = torch.empty(3 * ctx.N, device="cuda")
        _mm().mm_get_m(ctx, o)
        _mm().mm_sync(ctx)
        outs.append(o.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("grid", [(32, 32, 2), (20, 12, 3)])
def test_multi_step_graphs_are_bitwise_equal_to_direct_launches(monkeypatch, grid):
    """Runs of 37 then 16 steps: with graphs these take 16-step graphs (their
    steps chained by programmatic launch on the two-kernel path) plus, for
    the remainder, direct launches on the two-kernel path and single-step
    graphs from either parity elsewhere; the states must equal launch-by-
    launch stepping bit for bit."""
    cell = (5e-9, 5e-9, 3e-9)
    M = inputs.random_unit_m(grid, MS, seed=9)
    outs = []
    for flag in ("0", "1"):
        monkeypatch.setenv("MM_NO_GRAPHS", flag)
        ctx = _ctx(grid, cell, Ku=1e4, alpha=0.1)
        _mm().mm_set_field(ctx, (2e3, -1e3, 5e2))
        _mm().mm_set_m(ctx, _dev(M))
        _mm().mm_step(ctx, 37, 1e-13)
        _mm().mm_step(ctx, 16, 1e-13)
        o = torch.empty(3 * ctx.N, device="cuda")
        _mm().mm_get_m(ctx, o)
        _mm().mm_sync(ctx)
        outs.append(o.cpu().numpy())
    assert np.all(np.isfinite(outs[0]))
    assert np.array_equal(outs[0], outs[1])


def test_thin_film_32_random_start_1000_steps():
    """32x32x1 film, 5x5x3 nm, Ms 8.6e5, A 1.3e-11, Ku 0, alpha 0.5, random
    start (seed 1), H_ext 0, 1000 Euler steps of 1e-13 s, FP32 GPU vs FP64
    oracle: M within 1e-4, H_demag of the final state within 1e-5."""
    w = inputs.THIN_FILM_32
    grid, cell = w["grid"], w["cell"]
    M = inputs.random_unit_m(grid, w["Ms"], w["seed"])
    ctx = _ctx(grid, cell, Ms=w["Ms"], A=w["A"], Ku=w["Ku"], alpha=w["alpha"], gamma=w["gamma"])
    _mm().mm_set_m(ctx, _dev(M))
    _mm().mm_step(ctx, w["steps"], w["dt"])
    out = torch.empty(3 * ctx.N, device="cuda")
    _mm().mm_get_m(ctx, out)
    _mm().mm_sync(ctx)
    Kt, Lp = oracle_spectrum(grid, cell)
    ref = L.run_euler(M.astype(np.float64), w["steps"], w["dt"], cell, w["Ms"], w["A"], w["Ku"],
                      w["alpha"], w["gamma"], w["H_ext"], Kt, Lp)
    got = _host(out, grid)
    err = rel_l2(got, ref)
    print("thin film 32x32x1, 1000 steps: M rel L2 error %.3e" % err)
    assert err < 1e-4
    Hd = torch.empty_like(out)
    _mm().mm_demag_field(ctx, out, Hd)
    assert rel_l2(_host(Hd, grid), D.demag_fft(got, Kt, Lp)) < 1e-5


@pytest.mark.parametrize("grid", inputs.FILM_SWEEP_GRIDS)
def test_film_sweep_full_size(grid):
    """Size-sweep grids at full size: H_demag of a seeded random state and
    ten steps from the uniform +x start under the 170 degree field."""
    w = inputs.FILM_SWEEP
    cell = w["cell"]
    M = inputs.random_unit_m(grid, w["Ms"], seed=3)
    ctx = _ctx(grid, cell, Ms=w["Ms"], A=w["A"], Ku=w["Ku"], alpha=w["alpha"], gamma=w["gamma"])
    Md = _dev(M)
    Hd = torch.empty_like(Md)
    _mm().mm_demag_field(ctx, Md, Hd)
    Kt, Lp = oracle_spectrum(grid, cell)
    assert rel_l2(_host(Hd, grid), D.demag_fft(M.astype(np.float64), Kt, Lp)) < 1e-5
    M0 = inputs.uniform_m(grid, w["Ms"], w["start"])
    _mm().mm_set_m(ctx, _dev(M0))
    _mm().mm_set_field(ctx, w["H_ext"])
    _mm().mm_step(ctx, 10, w["dt"])
    out = torch.empty_like(Md)
    _mm().mm_get_m(ctx, out)
    _mm().mm_sync(ctx)
    ref = L.run_euler(M0.astype(np.float64), 10, w["dt"], cell, w["Ms"], w["A"], w["Ku"], w["alpha"],
                      w["gamma"], w["H_ext"], Kt, Lp)
    # measure the change from the start, which is what the step computes
    got = _host(out, grid)
    assert rel_l2(got - M0, ref - M0) < 1e-4


def test_direct_sum_samples_at_256x256x4():
    """Independent of any FFT: H_demag at sampled cells of the 256x256x4
    film by the direct sum of Eq. (12) with the tensor evaluated afresh."""
    grid, cell = (256, 256, 4), inputs.FILM_SWEEP["cell"]
    M = inputs.random_unit_m(grid, MS, seed=4)
    ctx = _ctx(grid, cell)
    Md = _dev(M)
    Hd = torch.empty_like(Md)
    _mm().mm_demag_field(ctx, Md, Hd)
    got = _host(Hd, grid)
    cells = [(0, 0, 0), (255, 255, 3), (128, 77, 1), (3, 200, 2)]
    ref = D.demag_at_cells(M.astype(np.float64), cell, cells)
    scale = np.max(np.abs(ref))
    for s, (i, j, k) in enumerate(cells):
        assert np.max(np.abs(got[:, k, j, i] - ref[s])) < 1e-5 * scale


def _sampled_cells_check(grid, w, M, cells, launches):
    """H_demag at `cells` by the direct sum of Eq. (12) (to 1e-5 of the
    largest sampled field), then one Euler step of Eq. (6) at those cells
    from the oracle's exchange, anisotropy and Zeeman terms and that H_demag,
    against the GPU's step in the plan the context picks for this grid (its
    launches per step asserted)."""
    cell = w["cell"]
    Ms, A, Ku, alpha, gamma, dt = w["Ms"], w["A"], w["Ku"], w["alpha"], w["gamma"], w["dt"]
    ctx = _ctx(grid, cell, Ms=Ms, A=A, Ku=Ku, alpha=alpha, gamma=gamma)
    assert _mm().mm_plan_info(ctx)[1] == launches
    Md = _dev(M)
    Hd = torch.empty_like(Md)
    _mm().mm_demag_field(ctx, Md, Hd)
    got = _host(Hd, grid)
    M64 = M.astype(np.float64)
    Href = D.demag_at_cells(M64, cell, cells)
    scale = np.max(np.abs(Href))
    for s, (i, j, k) in enumerate(cells):
        assert np.max(np.abs(got[:, k, j, i] - Href[s])) < 1e-5 * scale
    _mm().mm_set_m(ctx, Md)
    _mm().mm_set_field(ctx, w["H_ext"])
    _mm().mm_step(ctx, 1, dt)
    out = torch.empty_like(Md)
    _mm().mm_get_m(ctx, out)
    _mm().mm_sync(ctx)
    M1 = _host(out, grid)
    Hloc = L.h_exchange(M64, cell, Ms, A) + L.h_anisotropy(M64, Ms, Ku)
    for s, (i, j, k) in enumerate(cells):
        m = M64[:, k, j, i].reshape(3, 1, 1, 1)
        H = Hloc[:, k, j, i].reshape(3, 1, 1, 1) + Href[s].reshape(3, 1, 1, 1) + \
            np.asarray(w["H_ext"], np.float64).reshape(3, 1, 1, 1)
        n = m + dt * L.llg_rhs(m, H, Ms, alpha, gamma)
        n = (n * (Ms / np.sqrt(np.sum(n * n)))).reshape(3)
        change = n - m.reshape(3)
        # 1e-4 of the step, plus eight FP32 units in the last place of Ms for
        # the rounding of the stored FP32 state
        tol = 1e-4 * np.max(np.abs(change)) + 8 * float(np.spacing(np.float32(Ms)))
        assert np.max(np.abs((M1[:, k, j, i] - m.reshape(3)) - change)) < tol


def test_cube_128_sampled_cells_in_the_benchmarked_plan():
    """The N = 128 point of the cube curve at full size, in the plan that
    `bench.py --workload cube` times (split y / z / y kernels + x-step
    kernel, single-step graph)."""
    w = inputs.CUBE
    grid = (128, 128, 128)
    M = inputs.random_unit_m(grid, w["Ms"], w["seed"])
    _sampled_cells_check(grid, w, M, [(0, 0, 0), (127, 127, 127), (64, 31, 97)], 4)


@pytest.mark.parametrize("grid,cells,launches", [
    ((1024, 1024, 1), [(0, 0, 0), (1023, 511, 0), (300, 1023, 0)], 2),    # two-kernel step, two-row tiles
    ((256, 256, 64), [(0, 255, 63), (97, 13, 31)], 4),                     # split passes + x-step kernel
])
def test_precision_grids_sampled_cells(grid, cells, launches):
    """The precision workloads at full size (2.5 nm cells, the smooth
    perturbed start) in the plans their long runs use: direct-sum H_demag and
    one Euler step at sampled cells (the full 10k-step comparison is the
    opt-in precision study)."""
    w = dict(inputs.PRECISION)
    M = inputs.perturbed_m(grid, w["Ms"], w["seed"], w["amplitude"])
    _sampled_cells_check(grid, w, M, cells, launches)


@pytest.mark.parametrize("grid", [(24, 16, 3), (32, 32, 4)])
def test_energy_terms(grid):
    cell = (5e-9, 5e-9, 3e-9)
    Ku, Hext = 3e4, (2e4, -1e4, 5e3)
    M = inputs.random_unit_m(grid, MS, seed=13)
    ctx = _ctx(grid, cell, Ku=Ku)
    _mm().mm_set_field(ctx, Hext)
    _mm().mm_set_m(ctx, _dev(M))
    E = _mm().mm_energy(ctx)
    Kt, Lp = oracle_spectrum(grid, cell)
    M64 = M.astype(np.float64)
    ref = L.energy_terms(M64, D.demag_fft(M64, Kt, Lp), cell, MS, A_EX, Ku, Hext)
    scale = np.max(np.abs(ref[1:]))
    assert np.max(np.abs(E - ref)) < 1e-6 * scale


def test_norm_kept_and_energy_decays_on_gpu():
    grid, cell = (32, 32, 2), (5e-9, 5e-9, 3e-9)
    M = inputs.random_unit_m(grid, MS, seed=2)
    ctx = _ctx(grid, cell, Ku=5e2, alpha=0.5)
    _mm().mm_set_field(ctx, (1e4, 0.0, 0.0))
    _mm().mm_set_m(ctx, _dev(M))
    E_prev = _mm().mm_energy(ctx)[0]
    for _ in range(20):
        _mm().mm_step(ctx, 5, 1e-13)
        E = _mm().mm_energy(ctx)[0]
        assert E <= E_prev + 1e-7 * abs(E_prev)
        E_prev = E
    out = torch.empty(3 * ctx.N, device="cuda")
    _mm().mm_get_m(ctx, out)
    got = _host(out, grid)
    assert np.max(np.abs(np.sqrt(np.sum(got * got, axis=0)) - MS)) < 1e-6 * MS


def test_host_buffers_round_trip():
    grid, cell = (9, 7, 2), (5e-9, 5e-9, 3e-9)
    M = inputs.random_unit_m(grid, MS, seed=8).reshape(-1)
    ctx = _ctx(grid, cell)
    _mm().mm_set_m(ctx, np.ascontiguousarray(M))
    back = np.zeros_like(M)
    _mm().mm_get_m(ctx, back)
    assert np.array_equal(back, M)


def test_nonfinite_state_is_reported():
    grid, cell = (8, 8, 1), (5e-9, 5e-9, 3e-9)
    M = inputs.random_unit_m(grid, MS, seed=8)
    M[0, 0, 3, 3] = np.nan
    ctx = _ctx(grid, cell)
    _mm().mm_set_m(ctx, _dev(M))
    _mm().mm_step(ctx, 2, 1e-13)
    with pytest.raises(_mm().MMError) as e:
        _mm().mm_sync(ctx)
    assert e.value.code == _mm().MM_ENONFINITE
    # a fresh state clears the flag
    _mm().mm_set_m(ctx, _dev(inputs.random_unit_m(grid, MS, seed=9)))
    _mm().mm_step(ctx, 2, 1e-13)
    _mm().mm_sync(ctx)


def test_argument_errors_on_gpu():
    grid, cell = (8, 8, 1), (5e-9, 5e-9, 3e-9)
    ctx = _ctx(grid, cell)
    Md = _dev(inputs.random_unit_m(grid, MS, seed=1))
    with pytest.raises(_mm().MMError) as e:
        _mm().mm_demag_field(ctx, Md, Md)
    assert e.value.code == _mm().MM_EINVAL
    with pytest.raises(_mm().MMError):
        _mm().mm_step(ctx, 1, -1e-13)
    with pytest.raises(_mm().MMError) as e:
        _mm().mm_create((3000, 8, 1), cell, MS, A_EX, 0.0, 0.5, GAMMA)   # padded x length > 4096
    assert e.value.code == _mm().MM_EUNSUPPORTED


POW2_GRIDS = [(16, 16, 1), (32, 32, 2), (64, 64, 4), (256, 256, 4), (128, 64, 8), (16, 1024, 1),
              (1024, 16, 2), (512, 32, 1), (64, 512, 2), (32, 16, 8)]


@pytest.mark.parametrize("nofast", ["0", "1"])
@pytest.mark.parametrize("grid", POW2_GRIDS)
def test_power_of_two_paths_demag_and_steps(grid, nofast, monkeypatch):
    """The compile-time power-of-two kernels and the generic mixed-radix
    kernels must both match the oracle on the grids the former cover."""
    monkeypatch.setenv("MM_NO_FAST", nofast)
    cell = (4e-9, 4e-9, 3e-9)
    Ku, alpha, dt, Hext = 1e4, 0.1, 5e-14, (1e4, -5e3, 2e3)
    M = inputs.random_unit_m(grid, MS, seed=31)
    ctx = _ctx(grid, cell, Ku=Ku, alpha=alpha)
    Md = _dev(M)
    Hd = torch.empty_like(Md)
    _mm().mm_demag_field(ctx, Md, Hd)
    Kt, Lp = oracle_spectrum(grid, cell)
    M64 = M.astype(np.float64)
    Href = D.demag_fft(M64, Kt, Lp)
    assert rel_l2(_host(Hd, grid), Href) < 1e-5
    assert rel_max(_host(Hd, grid), Href) < 1e-5
    _mm().mm_set_field(ctx, Hext)
    _mm().mm_set_m(ctx, Md)
    _mm().mm_step(ctx, 3, dt)
    out = torch.empty_like(Md)
    _mm().mm_get_m(ctx, out)
    _mm().mm_sync(ctx)
    ref = L.run_euler(M64, 3, dt, cell, MS, A_EX, Ku, alpha, GAMMA, Hext, Kt, Lp)
    assert rel_l2(_host(out, grid), ref) < 1e-5


@pytest.mark.parametrize("grid", [(64, 32, 4), (48, 20, 3)])
def test_steps_interleaved_with_other_calls(grid):
    """Steps, field evaluations, energies and state changes in any order give
    the same trajectory as the oracle (the two-kernel step keeps the next
    step's spectrum between calls and must notice when it is stale)."""
    cell = (4e-9, 4e-9, 3e-9)
    Ku, alpha, dt, Hext = 2e4, 0.2, 5e-14, (2e4, 1e4, -3e3)
    M = inputs.random_unit_m(grid, MS, seed=41)
    M2 = inputs.random_unit_m(grid, MS, seed=42)
    ctx = _ctx(grid, cell, Ku=Ku, alpha=alpha)
    _mm().mm_set_field(ctx, Hext)
    _mm().mm_set_m(ctx, _dev(M))
    Kt, Lp = oracle_spectrum(grid, cell)
    ref = M.astype(np.float64)
    args = (dt, cell, MS, A_EX, Ku, alpha, GAMMA, Hext, Kt, Lp)
    scratch_in = _dev(M2)
    scratch_out = torch.empty_like(scratch_in)
    for n, action in ((3, "demag"), (2, "energy"), (1, "heff"), (4, "setm"), (2, None)):
        _mm().mm_step(ctx, n, dt)
        ref = L.run_euler(ref, n, *args)
        if action == "demag":
            _mm().mm_demag_field(ctx, scratch_in, scratch_out)
        elif action == "energy":
            _mm().mm_energy(ctx)
        elif action == "heff":
            _mm().mm_effective_field(ctx, scratch_in, scratch_out)
        elif action == "setm":
            _mm().mm_set_m(ctx, scratch_in)
            ref = M2.astype(np.float64)
    out = torch.empty_like(scratch_in)
    _mm().mm_get_m(ctx, out)
    _mm().mm_sync(ctx)
    assert rel_l2(_host(out, grid) - M2, ref - M2) < 1e-4
    assert rel_l2(_host(out, grid), ref) < 1e-6


THICK_GRIDS = [(8, 8, 9), (20, 12, 10), (16, 16, 16), (32, 32, 32), (24, 10, 12), (16, 32, 64), (32, 16, 128),
               (16, 512, 8), (16, 1024, 4)]


@pytest.mark.parametrize("grid", THICK_GRIDS)
def test_thick_samples_split_pass(grid):
    """nz > 8, or a kx plane too large for shared memory: pass 2 runs as
    separate y / z / y kernels (compile-time ones for power-of-two ny, nz)."""
    cell = (4e-9, 4e-9, 4e-9)
    M = inputs.random_unit_m(grid, MS, seed=51)
    ctx = _ctx(grid, cell, Ku=1e4, alpha=0.3)
    assert _mm().mm_plan_info(ctx)[1] in (4, 5)          # 4: compile-time split + x-step kernel
    Md = _dev(M)
    Hd = torch.empty_like(Md)
    _mm().mm_demag_field(ctx, Md, Hd)
    Kt, Lp = oracle_spectrum(grid, cell)
    M64 = M.astype(np.float64)
    Href = D.demag_fft(M64, Kt, Lp)
    assert rel_l2(_host(Hd, grid), Href) < 1e-5
    assert rel_max(_host(Hd, grid), Href) < 1e-5
    _mm().mm_set_m(ctx, Md)
    _mm().mm_step(ctx, 3, 5e-14)
    out = torch.empty_like(Md)
    _mm().mm_get_m(ctx, out)
    _mm().mm_sync(ctx)
    ref = L.run_euler(M64, 3, 5e-14, cell, MS, A_EX, 1e4, 0.3, GAMMA, (0, 0, 0), Kt, Lp)
    assert rel_l2(_host(out, grid), ref) < 1e-5


@pytest.mark.parametrize("method", ["heun", "rk4"])
@pytest.mark.parametrize("grid", [(20, 12, 3), (32, 32, 2), (64, 64, 4)])
def test_runge_kutta_steps_match_oracle(method, grid):
    cell = (4e-9, 4e-9, 3e-9)
    Ku, alpha, dt, Hext = 1e4, 0.2, 1e-13, (2e4, -1e4, 5e3)
    M = inputs.random_unit_m(grid, MS, seed=61)
    ctx = _ctx(grid, cell, Ku=Ku, alpha=alpha)
    _mm().mm_set_integrator(ctx, method)
    _mm().mm_set_field(ctx, Hext)
    _mm().mm_set_m(ctx, _dev(M))
    _mm().mm_step(ctx, 5, dt)
    out = torch.empty(3 * ctx.N, device="cuda")
    _mm().mm_get_m(ctx, out)
    _mm().mm_sync(ctx)
    Kt, Lp = oracle_spectrum(grid, cell)
    ref = L.run_rk(M.astype(np.float64), 5, dt, method, cell, MS, A_EX, Ku, alpha, GAMMA, Hext, Kt, Lp)
    got = _host(out, grid)
    assert rel_l2(got - M, ref - M) < 1e-4
    assert rel_l2(got, ref) < 1e-5
    # switching back to Euler gives the Euler trajectory again
    _mm().mm_set_integrator(ctx, "euler")
    _mm().mm_set_m(ctx, _dev(M))
    _mm().mm_step(ctx, 2, dt)
    _mm().mm_get_m(ctx, out)
    _mm().mm_sync(ctx)
    ref_e = L.run_euler(M.astype(np.float64), 2, dt, cell, MS, A_EX, Ku, alpha, GAMMA, Hext, Kt, Lp)
    assert rel_l2(_host(out, grid), ref_e) < 1e-5


def _random_grids(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        g = (int(rng.integers(1, 41)), int(rng.integers(1, 41)), int(rng.integers(1, 13)))
        if g[0] * g[1] * g[2] >= 2 and g not in out:
            out.append(g)
    return out


@pytest.mark.parametrize("grid", _random_grids(16, seed=2024) + [(16, 64, 12), (32, 16, 24), (64, 48, 2)])
def test_random_grid_sizes_demag_and_step(grid):
    """Seeded random sizes (every padded length the plan can pick, odd and
    prime extents, thin and thick samples, plus power-of-two and mixed cases):
    H_demag per evaluation and two Euler steps against the oracle."""
    cell = (4e-9, 3e-9, 2e-9)
    M = inputs.random_unit_m(grid, MS, seed=sum(grid) + 7)
    ctx = _ctx(grid, cell, Ku=2e4, alpha=0.2)
    _mm().mm_set_field(ctx, (1e4, -5e3, 2e3))
    Md = _dev(M)
    Hd = torch.empty_like(Md)
    _mm().mm_demag_field(ctx, Md, Hd)
    Kt, Lp = oracle_spectrum(grid, cell)
    M64 = M.astype(np.float64)
    Href = D.demag_fft(M64, Kt, Lp)
    assert rel_l2(_host(Hd, grid), Href) < 1e-5
    _mm().mm_set_m(ctx, Md)
    _mm().mm_step(ctx, 2, 2e-14)
    out = torch.empty_like(Md)
    _mm().mm_get_m(ctx, out)
    _mm().mm_sync(ctx)
    ref = L.run_euler(M64, 2, 2e-14, cell, MS, A_EX, 2e4, 0.2, GAMMA, (1e4, -5e3, 2e3), Kt, Lp)
    assert rel_l2(_host(out, grid) - M64, ref - M64) < 1e-4
    assert rel_l2(_host(out, grid), ref) < 1e-6


@pytest.mark.parametrize("grid", [(2048, 2, 1), (3, 2048, 1), (2, 3, 2048), (1025, 3, 2)])
def test_longest_padded_axes(grid):
    """The largest padded length the plan admits (4096) on each axis, and a
    smooth length above 2048 (1025 -> 2160): demag and one step against the
    oracle."""
    cell = (3e-9, 3e-9, 3e-9)
    M = inputs.random_unit_m(grid, MS, seed=77)
    ctx = _ctx(grid, cell, Ku=1e4, alpha=0.3)
    Md = _dev(M)
    Hd = torch.empty_like(Md)
    _mm().mm_demag_field(ctx, Md, Hd)
    Kt, Lp = oracle_spectrum(grid, cell)
    M64 = M.astype(np.float64)
    assert rel_l2(_host(Hd, grid), D.demag_fft(M64, Kt, Lp)) < 1e-5
    _mm().mm_set_m(ctx, Md)
    _mm().mm_step(ctx, 1, 2e-14)
    out = torch.empty_like(Md)
    _mm().mm_get_m(ctx, out)
    _mm().mm_sync(ctx)
    ref = L.run_euler(M64, 1, 2e-14, cell, MS, A_EX, 1e4, 0.3, GAMMA, (0, 0, 0), Kt, Lp)
    assert rel_l2(_host(out, grid) - M64, ref - M64) < 1e-4


def test_zero_and_negative_step_counts():
    """n = 0 leaves the state untouched bit for bit; n < 0 is rejected (bad
    create arguments are covered without a GPU in test_abi)."""
    grid, cell = (4, 4, 4), (3e-9, 3e-9, 3e-9)
    M = inputs.random_unit_m(grid, MS, seed=78)
    ctx = _ctx(grid, cell)
    _mm().mm_set_m(ctx, _dev(M))
    _mm().mm_step(ctx, 0, 1e-13)
    out = torch.empty(3 * ctx.N, device="cuda")
    _mm().mm_get_m(ctx, out)
    _mm().mm_sync(ctx)
    assert np.array_equal(out.cpu().numpy(), np.ascontiguousarray(M, np.float32).reshape(-1))
    with pytest.raises(_mm().MMError) as e:
        _mm().mm_step(ctx, -1, 1e-13)
    assert e.value.code == _mm().MM_EINVAL
