"""Plain FP64 CPU oracle for the Lamb-Helmholtz vortex FMM (test infrastructure).

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product library (``paper_1201_5430_gb300``) never imports, links or runs
anything here, and nothing here imports the product. The two share no code; the
only common module is ``workloads`` (seeded synthetic inputs, no method arithmetic).

Everything is written for a reader who checks it against the paper by eye:

* ``basis``       -- solid harmonics R_n^m, S_n^m (Eqs. rsbf1-rsbf7).
* ``operators``   -- translation maps (Eqs. mr2, mr3), differential operators
                     D_r, D_t, D_{r x t} (App. A, Eqs. dr1-drt7) and the R/S
                     conversions (Eqs. drt10, drt11).
* ``expansions``  -- P2M (Sec. 4.3: Eq. eve4, cross-checked by Eq. eve10) and
                     evaluation of local expansions (Sec. 4.5: Eqs. evf3, evf6).
* ``direct``      -- the exact smoothed Biot-Savart sum (Eqs. 1, 2, vem1, s1.1),
                     O(N*M) double loop in vectorised numpy ("O1").
* ``tree``        -- Morton keys, uniform octree, colleague and interaction lists.
* ``fmm``         -- the plain FP64 Lamb-Helmholtz FMM ("O2"), dense complex
                     translations, one conversion after every translation (Sec. 4).
* ``rk4``         -- classical RK4 time step of Eq. s1.1.
* ``complex_psi`` -- one complex FMM for Psi = phi + i chi (Sec. 4.2, Eq. chf1):
                     one complex translation per box pair, conversions on the
                     real potentials split from Psi.
* ``rcr``         -- rotation - coaxial translation - back rotation with the coaxial
                     conversions of Eq. rcr1 (Sec. 4.4).
* ``vfm``         -- vortex filament elements (Sec. 5.3, App. B): the closed-form
                     segment field (Eq. dis2), its Gauss-Legendre S-expansion
                     (Eqs. vf5-vf7) and the FMM with the nodes as receivers.
* ``scalar``      -- the paper's reference case (Sec. 5.2): phi and grad phi of
                     monopoles, direct ("O1s") and by the scalar harmonic FMM
                     over the same octree ("O2s").

Coefficient arrays are complex, full-m, unscaled (the paper's basis): an array
``c`` of shape (p, 2p-1) holds c_n^m at ``c[n, m + p - 1]`` for n < p, |m| <= n,
and zero elsewhere.
"""
