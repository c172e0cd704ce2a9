"""Plain CPU reference ("oracle") for the Mueller body-of-revolution solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  The product path (``paper_1810_07067_gb300``) never imports
it and shares no code with it.

Everything here is written from the paper's definitions in the plainest
form that is still fast enough for tests, in complex128:

* ``gauss``   - Gauss-Legendre rules, Lagrange interpolation and the near-panel
                support rules that define the Nystrom discretisation (Section 5).
* ``green``   - the modal Green's function g_m at k0 and k1, its first target
                derivatives and the second target derivatives of the k0-k1
                difference, by direct composite Gauss-Legendre quadrature of
                the unsplit integrands over phi (eqs. green11, firstder; no FFT,
                no kernel splitting).
* ``system``  - Lemma 1, the modal N and K operators and the Mueller system
                (eq. mullerrep), assembled mode by mode, with L2 weighting.
* ``linalg``  - naive partial-pivot LU and triangular solves.
* ``fields``  - modal plane-wave data (eq. pw) and far field (eq. farfieldform,
                with the M term as in eq. exteriorfield).
* ``mie``     - the Mie series for a dielectric sphere (textbook closed form).

Readings of the paper where it is garbled or silent are listed in the module
that applies them.
"""
