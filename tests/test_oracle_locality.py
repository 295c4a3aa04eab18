"""The reach of the oracle's step: with four ghost layers per side, k steps
of a block of the periodic domain depend only on the initial state within
4 k cells of it.  Stepping that neighbourhood k times, each step's interior
becoming the next step's ghosted input, reproduces the whole-domain run
bit for bit (the construction the 256^3 multi-step GPU parity test uses).
A stencil wider than the ghost layers, or a periodic fill read inside the
step, would break the equality."""
import numpy as np

import oracle as O
from paper_1110_0740_gb300 import workloads as W
from tests.test_gpu_error_table import _oracle_block, _wrap_block


def test_k_steps_of_a_block_from_its_domain_of_dependence():
    n, k, b = 32, 3, 4
    U0 = W.mhd_blast_3d(n, seed=3, kmax=3)
    dx = [1.0 / n] * 3
    dt, ch = O.dt_ch(O.mhd_max_speed(U0, [n] * 3, 3, dx), dx, 3, 0.3)
    U = U0.copy()
    for _ in range(k):
        O.fill_periodic(U, [n] * 3, 3)
        U, bad = O.mhd_step(U, [n] * 3, 3, dx, dt, ch, recon=1)
        assert bad == 0
    Ui, Uf = O.interior(U0, [n] * 3, 3), O.interior(U, [n] * 3, 3)
    for lo in ([5, 7, 9], [n - 2, 1, n - 3]):
        assert np.array_equal(_oracle_block(Ui, lo, b, k, dx, dt, ch), _wrap_block(Uf, lo, b))
