"""FP64 CPU oracle for the split-CTMRG hot path (test infrastructure only).

This package is the slow, plain reference that the CUDA path is checked against.
It is test infrastructure: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
product path (``paper_2502_10298_gb300``) never imports, links or runs it, and it
shares no code with that path; the only common module is ``ipeps_inputs`` (seeded
input generators, no method arithmetic).

Everything is written with plain PyTorch CPU ops in float64 so that autograd
provides an independent reference gradient.  Modules:

* ``svd``         -- full SVD with a Lorentzian-broadened backward.
* ``ctmrg``       -- initial environment, the split-CTMRG left move (ket stage with
                     green/yellow projectors, bra stage with teal/red projectors),
                     the conventional double-layer CTMRG with 2x2-patch projectors,
                     the frame maps that turn a left move into the other three
                     directions, and the directional sweep.
                     Also the run to a fixed point (``ctmrg_run``, corner spectra)
                     and separate environment / interlayer dimensions (``chi_pair``).
* ``energy``      -- 2x2-patch energy from the (fused) environment.
* ``statevector`` -- brute-force expectation values of small cluster states.
* ``fixed_point`` -- the energy gradient by implicit differentiation of the
                     converged environment.

Parity status: every function is pinned by ``tests/test_oracle_pins.py``.  The
teal/red rho networks follow a documented reading (their figures are missing
from the paper); they are pinned as parts of the method -- by the projector
identities, Onsager's exact correlator, the exactly solvable cluster states and
the split/conventional agreement -- while their literal match to the missing
figures cannot be checked.
"""
