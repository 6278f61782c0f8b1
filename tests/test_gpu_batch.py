"""Batched stepping of independent samples of uneven size (mm_batch_*):
each sample must follow its own FP64 oracle trajectory, and equal a
single-sample context run on the same generic kernels bit for bit."""
import numpy as np
import pytest

from oracle import llg as L
from paper_1406_7459_gb300 import inputs
from tests._helpers import oracle_spectrum, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _make(samples):
    from paper_1406_7459_gb300 import mm
    b = mm.mm_batch_create([s["grid"] for s in samples], [s["cell"] for s in samples],
                           [s["Ms"] for s in samples], [s["A"] for s in samples], [s["Ku"] for s in samples],
                           [s["alpha"] for s in samples], [s["gamma"] for s in samples])
    mm.mm_batch_set_field(b, [s["H_ext"] for s in samples])
    M = np.concatenate([s["M"].reshape(-1) for s in samples])
    mm.mm_batch_set_m(b, torch.from_numpy(M).cuda())
    return b


def test_batch_matches_oracle_and_single_contexts(monkeypatch):
    from paper_1406_7459_gb300 import mm
    samples = inputs.batch_samples(10, seed=7, nx=(16, 96), ny=(16, 40), nz=(1, 3))
    b = _make(samples)
    dt, n = 5e-14, 6
    mm.mm_batch_step(b, n, dt)
    out = torch.empty(b.total, device="cuda")
    mm.mm_batch_get_m(b, out)
    mm.mm_batch_sync(b)
    got = out.cpu().numpy()
    monkeypatch.setenv("MM_NO_FAST", "1")
    for i, s in enumerate(samples):
        g = s["grid"]
        mine = got[b.offsets[i]:b.offsets[i + 1]].reshape(3, g[2], g[1], g[0]).astype(np.float64)
        Kt, Lp = oracle_spectrum(g, s["cell"])
        ref = L.run_euler(s["M"].astype(np.float64), n, dt, s["cell"], s["Ms"], s["A"], s["Ku"], s["alpha"],
                          s["gamma"], s["H_ext"], Kt, Lp)
        assert rel_l2(mine, ref) < 1e-5, (i, g)
        ctx = mm.mm_create(g, s["cell"], s["Ms"], s["A"], s["Ku"], s["alpha"], s["gamma"])
        mm.mm_set_field(ctx, s["H_ext"])
        mm.mm_set_m(ctx, torch.from_numpy(s["M"].reshape(-1)).cuda())
        mm.mm_step(ctx, n, dt)
        one = torch.empty(3 * ctx.N, device="cuda")
        mm.mm_get_m(ctx, one)
        mm.mm_sync(ctx)
        assert np.array_equal(one.cpu().numpy(), got[b.offsets[i]:b.offsets[i + 1]]), (i, g)


def test_autotune_keeps_state_and_results():
    from paper_1406_7459_gb300 import mm
    samples = inputs.batch_samples(16, seed=9, nx=(16, 128), ny=(16, 48), nz=(1, 2))
    b = _make(samples)
    before = torch.empty(b.total, device="cuda")
    mm.mm_batch_get_m(b, before)
    choice, ms = mm.mm_batch_autotune(b, 5e-14)
    after = torch.empty(b.total, device="cuda")
    mm.mm_batch_get_m(b, after)
    assert torch.equal(before, after)
    assert choice[0] in (2, 4, 8) and choice[1] in (2, 4) and choice[2] in (128, 256)
    assert choice[3] in (1, 2, 4, 8)
    assert len(ms) == 16 and all(m > 0 for m in ms)
    mm.mm_batch_step(b, 3, 5e-14)
    mm.mm_batch_get_m(b, after)
    mm.mm_batch_sync(b)
    got = after.cpu().numpy()
    for i, s in enumerate(samples[:4]):
        g = s["grid"]
        Kt, Lp = oracle_spectrum(g, s["cell"])
        ref = L.run_euler(s["M"].astype(np.float64), 3, 5e-14, s["cell"], s["Ms"], s["A"], s["Ku"], s["alpha"],
                          s["gamma"], s["H_ext"], Kt, Lp)
        mine = got[b.offsets[i]:b.offsets[i + 1]].reshape(3, g[2], g[1], g[0])
        assert rel_l2(mine, ref) < 1e-5


def test_full_batch_workload_sampled(monkeypatch):
    """The benchmarked batch at full size: the 512 samples of the batch
    workload (seed 3), autotuned and stepped as one batch; four of them (the
    largest among them) checked against their FP64 oracle trajectories and,
    bit for bit, against single contexts on the same generic kernels."""
    from paper_1406_7459_gb300 import mm
    samples = inputs.batch_samples(512, seed=3)
    b = _make(samples)
    dt, n = 5e-14, 4
    choice, _ = mm.mm_batch_autotune(b, dt)
    mm.mm_batch_step(b, n, dt)
    out = torch.empty(b.total, device="cuda")
    mm.mm_batch_get_m(b, out)
    mm.mm_batch_sync(b)
    got = out.cpu().numpy()
    sizes = [s["grid"][0] * s["grid"][1] * s["grid"][2] for s in samples]
    picks = sorted({0, 255, 511, int(np.argmax(sizes))})
    monkeypatch.setenv("MM_NO_FAST", "1")
    for i in picks:
        s = samples[i]
        g = s["grid"]
        mine = got[b.offsets[i]:b.offsets[i + 1]]
        Kt, Lp = oracle_spectrum(g, s["cell"])
        ref = L.run_euler(s["M"].astype(np.float64), n, dt, s["cell"], s["Ms"], s["A"], s["Ku"], s["alpha"],
                          s["gamma"], s["H_ext"], Kt, Lp)
        assert rel_l2(mine.reshape(3, g[2], g[1], g[0]).astype(np.float64), ref) < 1e-5, (i, g)
        ctx = mm.mm_create(g, s["cell"], s["Ms"], s["A"], s["Ku"], s["alpha"], s["gamma"])
        mm.mm_set_field(ctx, s["H_ext"])
        mm.mm_set_m(ctx, torch.from_numpy(s["M"].reshape(-1)).cuda())
        mm.mm_step(ctx, n, dt)
        one = torch.empty(3 * ctx.N, device="cuda")
        mm.mm_get_m(ctx, one)
        mm.mm_sync(ctx)
        assert np.array_equal(one.cpu().numpy(), mine), (i, g, choice)


def _run_path(samples, path, runs, dt=5e-14, autotune=False):
    from paper_1406_7459_gb300 import mm
    b = _make(samples)
    if autotune:
        mm.mm_batch_autotune(b, dt)
    mm.mm_batch_set_path(b, path)
    for n in runs:
        mm.mm_batch_step(b, n, dt)
    out = torch.empty(b.total, device="cuda")
    mm.mm_batch_get_m(b, out)
    mm.mm_batch_sync(b)
    return out.cpu().numpy()


def test_persistent_batch_is_bitwise_the_graph_batch():
    """One cooperative launch per call, (sample, tile) items taken from a
    work queue per pass, against the three batched kernels per step of the
    graph path: runs of 1, 3 and 6 steps (the spectra carried from one call to
    the next) give the same bits."""
    from paper_1406_7459_gb300 import mm
    samples = inputs.batch_samples(10, seed=7, nx=(16, 96), ny=(16, 40), nz=(1, 3))
    a = _run_path(samples, mm.MM_STEP_PERSISTENT, (1, 3, 6))
    b = _run_path(samples, mm.MM_STEP_GRAPH, (1, 3, 6))
    assert np.all(np.isfinite(a))
    assert np.array_equal(a, b)


def test_persistent_batch_replays_one_captured_launch():
    """The persistent step is one cooperative launch per call captured in a
    CUDA graph: calls of 3, 3, 1 and 3 steps (the second and fourth replay
    a launch captured before, the third is captured anew) run from a graph
    and give the bits of the graph path."""
    from paper_1406_7459_gb300 import mm
    samples = inputs.batch_samples(6, seed=11, nx=(16, 80), ny=(16, 32), nz=(1, 2))
    runs = (3, 3, 1, 3)
    b = _make(samples)
    mm.mm_batch_set_path(b, mm.MM_STEP_PERSISTENT)
    assert mm.mm_batch_launch_form(b) == -1
    for n in runs:
        mm.mm_batch_step(b, n, 5e-14)
        assert mm.mm_batch_launch_form(b) == 1
    out = torch.empty(b.total, device="cuda")
    mm.mm_batch_get_m(b, out)
    mm.mm_batch_sync(b)
    ref = _run_path(samples, mm.MM_STEP_GRAPH, runs)
    assert np.array_equal(out.cpu().numpy(), ref)


def test_persistent_full_batch_workload_is_bitwise_the_graph_batch():
    """The benchmarked 512-sample batch, autotuned, four steps both ways."""
    from paper_1406_7459_gb300 import mm
    samples = inputs.batch_samples(512, seed=3)
    a = _run_path(samples, mm.MM_STEP_PERSISTENT, (4,), autotune=True)
    b = _run_path(samples, mm.MM_STEP_GRAPH, (4,), autotune=True)
    assert np.array_equal(a, b)


def test_persistent_batch_wait_gives_up_and_recovers():
    """A poll limit of 0: the grid-barrier waits give up at once and
    mm_batch_sync reports MM_ETIMEOUT (no GPU fault).  After the limit is
    restored and the state set again, the batch steps as the graph path."""
    from paper_1406_7459_gb300 import mm
    samples = inputs.batch_samples(10, seed=8, nx=(16, 96), ny=(16, 40), nz=(1, 2))
    b = _make(samples)
    mm.mm_batch_set_path(b, mm.MM_STEP_PERSISTENT)
    mm.mm_batch_set_wait_limit(b, 0)
    mm.mm_batch_step(b, 3, 5e-14)
    with pytest.raises(mm.MMError) as e:
        mm.mm_batch_sync(b)
    assert e.value.code == mm.MM_ETIMEOUT
    mm.mm_batch_set_wait_limit(b, 1 << 20)
    M = np.concatenate([s["M"].reshape(-1) for s in samples])
    mm.mm_batch_set_m(b, torch.from_numpy(M).cuda())
    mm.mm_batch_step(b, 3, 5e-14)
    out = torch.empty(b.total, device="cuda")
    mm.mm_batch_get_m(b, out)
    mm.mm_batch_sync(b)
    ref = _run_path(samples, mm.MM_STEP_GRAPH, (3,))
    assert np.array_equal(out.cpu().numpy(), ref)
    with pytest.raises(mm.MMError) as e:
        mm.mm_batch_set_path(b, 9)
    assert e.value.code == mm.MM_EINVAL
