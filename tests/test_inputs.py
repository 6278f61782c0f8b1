"""The seeded input recipes (paper_1406_7459_gb300/inputs.py), the one module
both the oracle and the GPU path read: each workload has the sizes, material
and distributions it is defined with, and the generators give unit-length
states scaled to Ms, reproducibly from their seeds."""
import numpy as np

from paper_1406_7459_gb300 import inputs

MS = 8.6e5


def _norms(M):
    return np.sqrt(np.sum(M.astype(np.float64) ** 2, axis=0))


def test_random_unit_states_have_length_ms_and_repeat_from_the_seed():
    a = inputs.random_unit_m((24, 20, 3), MS, seed=4)
    assert a.dtype == np.float32 and a.shape == (3, 3, 20, 24)
    assert np.max(np.abs(_norms(a) - MS)) < 1e-6 * MS
    assert np.array_equal(a, inputs.random_unit_m((24, 20, 3), MS, seed=4))
    assert not np.array_equal(a, inputs.random_unit_m((24, 20, 3), MS, seed=5))
    # directions spread over the sphere: each component's mean is near 0
    m = a.reshape(3, -1) / MS
    assert np.all(np.abs(m.mean(axis=1)) < 0.06)


def test_uniform_and_perturbed_states():
    u = inputs.uniform_m((8, 4, 2), MS)
    assert np.all(u[0] == np.float32(MS)) and np.all(u[1:] == 0)
    p = inputs.perturbed_m((32, 16, 2), MS, seed=2, amplitude=0.1)
    assert np.max(np.abs(_norms(p) - MS)) < 1e-6 * MS
    cosang = p[0].astype(np.float64) / MS
    assert 0.9 < cosang.min() and cosang.mean() > 0.99


def test_field_at_170_degrees():
    h = inputs.field_at_angle(2.5e4, 170.0)
    assert abs(np.hypot(h[0], h[1]) - 2.5e4) < 1e-9 * 2.5e4 and h[2] == 0.0
    assert abs(np.degrees(np.arctan2(h[1], h[0])) - 170.0) < 1e-9


def test_workload_recipes():
    t = inputs.THIN_FILM_32
    assert t["grid"] == (32, 32, 1) and t["cell"] == (5e-9, 5e-9, 3e-9)
    assert (t["Ms"], t["A"], t["Ku"], t["alpha"], t["gamma"]) == (8.6e5, 1.3e-11, 0.0, 0.5, 2.211e5)
    assert t["H_ext"] == (0.0, 0.0, 0.0) and t["dt"] == 1e-13 and t["steps"] == 1000 and t["seed"] == 1
    assert inputs.FILM_SWEEP_GRIDS == ((64, 64, 4), (128, 128, 4), (256, 256, 4), (512, 512, 8), (200, 60, 3))
    f = inputs.FILM_SWEEP
    assert f["cell"] == (4e-9, 4e-9, 4e-9) and f["Ku"] == 5e2 and f["alpha"] == 0.02
    assert f["start"] == (1.0, 0.0, 0.0) and f["H_ext"] == inputs.field_at_angle(2.5e4, 170.0)
    assert inputs.PRECISION_GRIDS == ((1024, 1024, 1), (256, 256, 64))
    p = inputs.PRECISION
    assert p["cell"] == (2.5e-9, 2.5e-9, 2.5e-9) and p["steps"] == 10000 and p["dt"] == 5e-14
    assert inputs.CUBE_SIZES == (8, 16, 32, 64, 128) and inputs.CUBE["cell"] == (4e-9, 4e-9, 4e-9)


def test_batch_of_512_samples_follows_its_distributions():
    """512 samples, seed 3: nx ~ U{16..256}, ny ~ U{16..64}, nz ~ U{1, 2},
    Ku ~ U[0, 1e4], |H_ext| ~ U[0, 5e4] in a uniformly random direction,
    alpha ~ U[0.01, 0.5]; each within its range, spread over it (means of
    the uniform laws within ~4 standard errors), reproducible."""
    s = inputs.batch_samples(512, seed=3)
    assert len(s) == 512
    g = np.array([x["grid"] for x in s])
    assert g[:, 0].min() >= 16 and g[:, 0].max() <= 256
    assert g[:, 1].min() >= 16 and g[:, 1].max() <= 64
    assert set(g[:, 2]) == {1, 2}
    ku = np.array([x["Ku"] for x in s])
    al = np.array([x["alpha"] for x in s])
    h = np.array([x["H_ext"] for x in s])
    hm = np.linalg.norm(h, axis=1)
    assert ku.min() >= 0 and ku.max() <= 1e4
    assert al.min() >= 0.01 and al.max() <= 0.5
    assert hm.max() <= 5e4

    def near(v, lo, hi):
        se = (hi - lo) / np.sqrt(12.0 * len(v))
        return abs(v.mean() - 0.5 * (lo + hi)) < 4 * se

    assert near(g[:, 0].astype(float), 16, 256) and near(g[:, 1].astype(float), 16, 64)
    assert near(ku, 0, 1e4) and near(al, 0.01, 0.5) and near(hm, 0, 5e4)
    d = h / hm[:, None]
    assert np.all(np.abs(d.mean(axis=0)) < 4 / np.sqrt(3 * 512))
    for x in s[:16]:
        assert x["M"].shape == (3, x["grid"][2], x["grid"][1], x["grid"][0])
        assert np.max(np.abs(_norms(x["M"]) - x["Ms"])) < 1e-6 * x["Ms"]
    again = inputs.batch_samples(512, seed=3)
    assert all(a["grid"] == b["grid"] and a["Ku"] == b["Ku"] for a, b in zip(s, again))
