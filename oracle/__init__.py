"""FP64 CPU oracle for HOTRG on 2D classical lattice models and quantum chains.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls, links or
executes anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py`` may use it.  It shares no
code, constants or helpers with the CUDA library in ``paper_2602_05900_gb300``.

Contents
--------
``hotrg``       plain FP64 NumPy HOTRG (initial tensors, X/Y coarse-graining
                steps, max-norm rescale, free energy).  Z = Tr T^N is Eq. (2) of
                the paper (Sec. II.A); the truncation by a higher-order SVD that is
                reduced to a matrix SVD / Hermitian eigendecomposition of a
                reshaped matrix follows Sec. II.A and Eq. (5).
``exact``       exact ln Z of small periodic lattices by a row transfer matrix.
``brute``       ctypes loader for ``brute_force.c`` (plain C enumeration of all
                spin configurations of a small torus).
``onsager``     Onsager's closed form of the 2D Ising free energy at h = 0.
``heisenberg``  quantum HOTRG of the spin-1/2 XXZ chain: the Trotterised
                imaginary-time cell tensor (Sec. II.A-B), dense small-chain
                references, and the schedule Y steps -> time trace -> X steps.
``itebd``       iTEBD ground state of the XXZ chain (Sec. II.A, Eq. 1): two-site
                gate updates with SVD truncation, bond and site energies.
``sampled``     element-by-element evaluation of single-step outputs, for checks
                at sizes where the full oracle is too slow.

Pins (what fixes each function independently of itself) are listed in the
module docstrings and exercised by ``tests/test_oracle_*.py``.
"""
