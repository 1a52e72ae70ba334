"""FP64 CPU oracle for real-space exact exchange, ACE and the TDA Casida matrix.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously correct statement of
what the GPU library computes.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the CUDA
path (``paper_2405_01522_gb300``) and never imports it; both sides only share the
seeded synthetic-input generator, which holds none of the method's arithmetic.

Paper: Panta & Strubbe, "Implementation of time-dependent Hartree-Fock in real
space" (arXiv 2405.01522).  Equation numbers follow the paper's order:
Eq. 2 exchange operator (Sec. 2), Eqs. 3-5 full linear-response problem, Eq. 7 RHF
matrix (Sec. 2), Eqs. 8-10 transition dipoles, oscillator strengths and strength
function (Sec. 2), Eqs. 11-13 ACE (Sec. 3.1), Eqs. 14-15 linear mixing and the relative
density error of the SCF cycle (Secs. 3.2, 3.4).

Modules
-------
coulomb   discrete Coulomb kernel and the isolated Poisson solve (FFT and direct sum)
exchange  pair densities, exact-exchange action, exchange / Hartree energies
ace       adaptively compressed exchange: build and apply
casida    coupling matrices K and K_d, TDA matrix, eigen-solve; the spin-polarised
          (UHF) coupling over alpha and beta transitions and its TDA matrix
eigensolver  FD4 Hamiltonian, kinetic-energy preconditioner, Rayleigh-Ritz step, and the
          3-layer conv3d network of the learned preconditioner with its gradients
spectra   dipole matrix elements, oscillator strengths, Lorentzian strength function,
          full (non-Tamm-Dancoff) TDHF in the half-size form and as the 2n x 2n problem
scf       closed-shell Hartree-Fock SCF on small grids, with ACE or exact exchange

Parity status: every public function here is pinned by ``tests/test_oracle_pins.py``
against closed forms, brute-force sums or invariants; none is "parity unpinned".
"""
from .coulomb import (C0, kernel_samples, kernel_spectrum, poisson_fft,
                      poisson_direct, potential_at)
from .exchange import (pair_density, exchange_apply, exchange_apply_at, exchange_apply_bruteforce,
                       exchange_energy, hartree_energy, inner)
from .ace import ace_build, ace_apply
from .casida import (transition_densities, casida_K, casida_K_bruteforce, casida_Kd,
                     tda_matrix, tda_solve, uhf_K, uhf_tda_matrix, HARTREE_EV)

__all__ = [
    "C0", "kernel_samples", "kernel_spectrum", "poisson_fft", "poisson_direct", "potential_at",
    "pair_density", "exchange_apply", "exchange_apply_at", "exchange_apply_bruteforce", "exchange_energy",
    "hartree_energy", "inner", "ace_build", "ace_apply", "transition_densities",
    "casida_K", "casida_K_bruteforce", "casida_Kd", "tda_matrix", "tda_solve",
    "uhf_K", "uhf_tda_matrix", "HARTREE_EV",
]
