"""FP64 CPU oracle for the demag + LLG hot path (test infrastructure only).

This package is the plain, slow, obviously correct statement of what the
GPU path computes.  It is TEST INFRASTRUCTURE: only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline`` /
``--impl reference`` legs may import it.  The product path
(``paper_1406_7459_gb300``) never imports it and shares no code with it.

Modules
  tensor  -- Newell cell-averaged demag tensor (Sec. 2, Eqs. (7), (11)-(12);
             the formula itself is deferred by the paper to its ref. [11]),
             Aharoni's prism factor (used only as an independent pin).
  demag   -- demag field by brute-force summation (Eq. (11)/(12)) and by the
             zero-padded FFT convolution (Eqs. (8)-(10), (13)-(16)).
  llg     -- exchange (Eqs. (3)-(4)), anisotropy (Eq. (5)), Zeeman, LLG
             right-hand side (Eq. (6)), forward Euler + renormalisation,
             Heun and classic RK4 steps, energy (Eq. (1)), macrospin
             closed form.

All arithmetic is float64.  Every function is pinned by a ``-m "not gpu"``
test against something other than itself (closed forms, brute force,
invariants); no function here is "parity unpinned".
"""
from .tensor import (newell_f, newell_g, newell_tensor, quadrature_tensor,
                     demag_tensor, tensor_octant, tensor_full_offsets,
                     aharoni_factor, MU0)
from .demag import (wrap_pad_kernel, kernel_spectrum, demag_fft, demag_brute,
                    demag_at_cells)
from .llg import (h_exchange, h_anisotropy, h_effective, llg_rhs, euler_step,
                  run_euler, rk_step, run_rk, energy_terms, macrospin_closed_form)
