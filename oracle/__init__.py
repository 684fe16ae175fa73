"""CPU FP64 oracle for the AIM-accelerated EFIE method of moments.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import this package.  The
library in ``paper_1010_1456_gb300`` never imports, links or runs it, and this
package imports nothing from the library: the two share no code.  The only
common input is ``aim_inputs`` (meshes and excitations, none of the method's
arithmetic).

Contents (paper: Wei & Yilmaz, "A Hybrid Parallelization of AIM for
Multi-Core Clusters", Sections 2.1-2.2 and 4.1, eq. 1):

* ``quadrature``  collapsed Gauss-Legendre triangle rules
* ``rwg``         RWG basis functions on triangle meshes (Section 2.1 meshes)
* ``efie``        EFIE Galerkin entries with singularity extraction, dense Z
* ``mfie``        MFIE Galerkin entries, CFIE, differentiated AIM weights
* ``aim``         AIM: moment-matching projection, grid Green's function
                  convolution, interpolation, near-zone correction (Section 2.2)
* ``excitation``  plane-wave right-hand side
* ``solve``       diagonally preconditioned GMRES(m), dense LU (Section 2.2)
* ``rcs``         bistatic RCS and err_theta-theta (eq. 1)
* ``mie``         Mie series for the PEC sphere (Section 2.2 reference)

Parity status of each function is stated in its docstring; all pins are in
``tests/test_oracle_*.py``.
"""

ETA0 = 376.730313668  # free-space impedance, ohm
