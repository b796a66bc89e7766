"""FP64 CPU oracle for the stochastic spin-coherent-state trace.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything here.  The product path
(the CUDA library and its Python binding) never imports, links or runs it, and
this package shares no code, table or constant with that path.

What it computes (Lewis, Fay and Manolopoulos, "An efficient quantum mechanical
method for radical pair recombination reactions"):

* ``spin``      -- Hamiltonian of Eq. 1, Haberkorn operator of Eq. 2 and the
                   singlet / triplet projectors of Eqs. 3-4 as dense matrices.
* ``philox``    -- the Philox4x32-10 counter-based generator (Salmon et al.,
                   SC'11), used to draw the coherent-state directions.
* ``coherent``  -- spin coherent states (Eq. 15) built literally as
                   cos^{2J}(theta/2) exp(tan(theta/2) e^{i phi} J_-) |J, J>,
                   and the sample initial states |S> x prod_k |Omega_k> (Eq. 19).
* ``dense``     -- the exact truncated yields by Van Loan's block exponential:
                   per-sample phi_S (Eq. 22 truncated at T), the deterministic
                   trace (Eq. 14) and the stochastic estimate (Eq. 18, Eq. 23).
* ``chebyshev`` -- a matrix-free FP64 Chebyshev propagator with an exact
                   per-step time integral for systems too large for ``dense``.

Pins (tests/test_oracle_*.py): closed forms for one spin-1/2 and one spin-1
nucleus, the nucleus-free singlet, norm decay, conservation, field-reversal
symmetry, Eq. 16, Eq. 17 by quadrature, unbiasedness, the effective hyperfine
fields printed for Table I (Eq. 21), brute-force time quadrature, and
agreement of the matrix-free path with the dense path.
"""
