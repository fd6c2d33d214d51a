"""FP64 CPU oracle for the PSATD step and its FDTD comparators.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) imports, calls or links anything in this package; only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.

The oracle is a plain, slow, obviously-correct restatement of what the paper
(Blaclard, Vincenti, Lehe, Vay 2016, "Pseudo-spectral Maxwell solvers for an
accurate modeling of Doppler harmonic generation on plasma mirrors with
Particle-In-Cell codes") says the solvers compute:

* ``psatd``      -- the pseudo-spectral analytical time-domain step (Sec. III.B,
                    item 2; Table 1 row "PSATD"): Maxwell's equations solved
                    exactly in (k, t) space under the assumption that the sources
                    are constant over one time step.
* ``fdtd``       -- the Yee and Cole-Karkkainen(-Cowan) finite-difference
                    solvers (Sec. III.A; Table 1 rows "Yee" and "CKC").
* ``dispersion`` -- the vacuum refractive index of each solver (Table 1), the
                    Snell-Descartes refraction toy model (Sec. IV.A, Eq. Snell)
                    and the closed forms of Appendix A.
* ``local``      -- the local-FFT decomposition (Sec. II.A.3): patches with
                    guard cells refreshed from their neighbours, each advanced as
                    a periodic domain of its own.
* ``farfield``   -- the Fraunhofer far-field transform of a field snapshot
                    (Sec. II.B), the diagnostic of the angularly resolved
                    harmonic spectrum.
``psatd`` also holds the staggered order-p variant (Table 1 row PSATD-p) and the
PSTD scheme (Table 1 row PSTD).

It shares no code with the CUDA path.  All floating point is FP64 (numpy).
"""
