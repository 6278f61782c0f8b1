"""Precision study on the large grids: FP32 GPU path against the FP64
oracle.  Long (minutes of oracle time), so it runs only with
MM_PRECISION_STUDY=1; it prints the error of each result as a number.

Film 1024x1024x1 and block 256x256x64, 2.5 nm cells, Ms 8.6e5, A 1.3e-11,
Ku 0, alpha 0.5, smooth start (+x with a seed-2 perturbation of 0.1,
renormalised), no field, Euler dt 5e-14 s.  H_demag error on the start
state and, for the film, on the GPU state every 1000 of 10k steps (the
oracle evaluates H on the same state); M error after as many steps as the
oracle can take in about a minute."""
import os
import time

import numpy as np
import pytest

from oracle import tensor as T, demag as D, llg as L
from paper_1406_7459_gb300 import inputs
from tests._helpers import rel_l2, rel_max

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.skipif(os.environ.get("MM_PRECISION_STUDY") != "1",
                                                   reason="set MM_PRECISION_STUDY=1")]


def _run(grid, total_steps, every, m_steps):
    from paper_1406_7459_gb300 import mm
    w = inputs.PRECISION
    cell = w["cell"]
    M0 = inputs.perturbed_m(grid, w["Ms"], w["seed"], w["amplitude"])
    t0 = time.time()
    Kt = D.kernel_spectrum(T.tensor_octant(grid, cell), D.default_lengths(grid))
    Lp = D.default_lengths(grid)
    t_setup = time.time() - t0
    ctx = mm.mm_create(grid, cell, w["Ms"], w["A"], w["Ku"], w["alpha"], w["gamma"])
    Md = torch.from_numpy(M0.reshape(-1)).cuda()
    mm.mm_set_m(ctx, Md)
    Hd = torch.empty_like(Md)
    nx, ny, nz = grid
    herr = []
    state = torch.empty_like(Md)
    done = 0
    while True:
        mm.mm_get_m(ctx, state)
        mm.mm_demag_field(ctx, state, Hd)
        torch.cuda.synchronize()
        Mh = state.cpu().numpy().reshape(3, nz, ny, nx).astype(np.float64)
        ref = D.demag_fft(Mh, Kt, Lp)
        got = Hd.cpu().numpy().reshape(3, nz, ny, nx)
        herr.append((done, rel_l2(got, ref), rel_max(got, ref)))
        if done >= total_steps:
            break
        mm.mm_step(ctx, every, w["dt"])
        done += every
    mm.mm_sync(ctx)
    # M after m_steps from the start, GPU vs oracle
    mm.mm_set_m(ctx, Md)
    mm.mm_step(ctx, m_steps, w["dt"])
    mm.mm_get_m(ctx, state)
    mm.mm_sync(ctx)
    t1 = time.time()
    Mref = L.run_euler(M0.astype(np.float64), m_steps, w["dt"], cell, w["Ms"], w["A"], w["Ku"], w["alpha"],
                       w["gamma"], w["H_ext"], Kt, Lp)
    t_oracle = time.time() - t1
    got = state.cpu().numpy().reshape(3, nz, ny, nx)
    merr = (rel_l2(got, Mref), rel_l2(got - M0, Mref - M0))
    print("\nPRECISION grid=%s H_demag rel L2 / rel max at steps %s; M after %d steps: rel L2 %.3e, "
          "rel L2 of the change %.3e (oracle set-up %.0f s, %d oracle steps %.0f s)"
          % (grid, ["%d: %.2e / %.2e" % h for h in herr], m_steps, merr[0], merr[1], t_setup, m_steps, t_oracle))
    return herr, merr


def test_film_1024x1024x1():
    herr, merr = _run((1024, 1024, 1), 10000, 1000, 40)
    assert all(h[1] < 1e-5 for h in herr)
    assert merr[0] < 1e-5


def test_block_256x256x64():
    herr, merr = _run((256, 256, 64), 0, 1000, 5)
    assert all(h[1] < 1e-5 for h in herr)
    assert merr[0] < 1e-5
