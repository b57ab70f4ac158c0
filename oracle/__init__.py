"""Plain, slow FP64 CPU oracle of the FFT phase-field-fracture toughness method (arXiv 2508.07424).

TEST INFRASTRUCTURE ONLY. Nothing on the product path imports this package: only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``
may use it. It shares no code with the CUDA library; both read their inputs from the seeded
generators in ``synth``.

Modules
-------
spectral   frequency vectors, spectral gradient/divergence and the Fourier-Galerkin operator G^
           of Eq. (GFourier), all on full complex FFTs of the whole grid.
material   stiffness tensors (cubic, isotropic), the rotation of Eq. (Crot), the cleavage tensor
           of Eq. (PFFani), degradation g of Sec. 2.1 and the spectral energy split.
solver     mechanics CG, damage CG, the dissipation (arc-length) control of Eq. (SystemDisany),
           crack-tip enrichment of Eqs. (damini)-(HistoryNumIni), toughness of Eqs. (JaviGc)-(ABC).
residuals  independent evaluation of the residuals R1, R2, R3 of Eq. (aniSystem_CrackLength).

Parity status: every function is pinned by a ``-m "not gpu"`` test (tests/test_oracle_*.py)
against closed forms, brute force, textbook results or invariants; see the test docstrings.
"""
