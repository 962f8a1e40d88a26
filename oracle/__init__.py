"""Plain, slow, obviously-correct CPU oracle for the Fresnel areal-quadrature method.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, links or runs
anything in this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.  It
shares no code, header, table or helper with the CUDA library in
``paper_2010_05978_gb300/csrc``; the only thing both sides see are the seeded
inputs produced by ``workloads.py`` (which holds none of the method's
arithmetic).

Contents (each function cites the passage of Barnett, "Efficient high-order
accurate Fresnel diffraction via areal quadrature and the nonuniform FFT",
arXiv:2010.05978, that it follows):

* ``quadrature``   -- Gauss-Legendre rules, vector line rules on the boundary,
                      the "dilation" areal rule (Sec. 3.1, eqs. aqnod/aqwei),
                      the periodic trapezoid line rule (eq. ptr).
* ``direct``       -- the direct O(NM) sum of eq. faq (unsplit form) and the
                      non-singular line integral NSLI (Appendix, eq. nsli),
                      in C with OpenMP (``oracle/direct.c``), FP64.
* ``closed_forms`` -- closed forms used to pin the oracle: disc on axis
                      (Appendix eq. dauger with R(theta) = R), the disc off
                      axis (radially symmetric Hankel reduction of eq. fres),
                      exact areas and moments, and brute-force adaptive 2D
                      integration of eq. fres on tiny cases.
* ``field``        -- the whole field u^ap / u^oc = 1 - u^ap (eq. bab) for a
                      list of panel families, built only from the above.
* ``gradient``     -- a starshade loss (mean |u^oc|^2 over kept targets and
                      problems) and its gradient with respect to the
                      B-spline petal profile, by differentiating the direct
                      sum of eq. faq by hand (adjoint sums in direct.c).

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
against closed forms, invariants or brute force; none is "parity unpinned".
"""
from . import quadrature, closed_forms  # noqa: F401
from .field import field, nodes, grid_targets  # noqa: F401
