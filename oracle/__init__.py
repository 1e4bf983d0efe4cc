"""Plain FP64 CPU oracle of the ternary "2f1s" phase-field lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import anything here.  The
CUDA library never calls into this package and this package never calls into
the CUDA library; they share no code, tables or constants.

The oracle follows Zhan, Chai and Shi, "A ternary phase-field model for
two-phase flows in complex geometries" (arXiv 2311.05091):

* ``lattice``     -- velocity sets, weights, natural-moment matrix M0 and the
                     Hermite lower-triangular matrix N (Appendix A).
* ``model``       -- the spreading coefficients gamma_p from Young's law and the
                     k(theta, kappa) closure (Sec. 2.2, Eq. kk), relaxation
                     rates (Sec. 3).
* ``lbm``         -- one coupled time step: isotropic stencils, chemical
                     potential, CH and NS Hermite-moment collisions, streaming
                     with half-way bounce-back (Sec. 2, Sec. 3).
* ``observables`` -- mass, Laplace pressure, droplet height and contact angle
                     (Sec. 4.2, 4.3).

Parity status per function is stated in each module header.
"""
