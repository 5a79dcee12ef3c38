"""Pins of the oracle's small-deformation theory (Section 3 and the Appendix)."""
import os

import numpy as np
from scipy.special import eval_legendre

from oracle import spt

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_quadrupole.txt")


def table2():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                drop, ca, e1, e2 = line.split()
                rows.append((drop, float(ca), float(e1) / 100.0, float(e2) / 100.0))
    return rows


def test_deformation_number_matches_the_shape_it_describes():
    """Eq. def_num against D = (r(0) - r(pi/2)) / (r(0) + r(pi/2)) evaluated on the shape
    r = 1 + Ca sum F^(1)_n P_n + Ca^2 sum F^(2)_n P_n (Legendre values from scipy): the two agree to
    O(Ca^3) for arbitrary mode amplitudes, which fixes every coefficient of Eq. def_num."""
    rng = np.random.default_rng(3)
    F1 = {2: rng.uniform(-1, 1), 4: rng.uniform(-1, 1)}
    F2 = {n: rng.uniform(-1, 1) for n in (2, 4, 6, 8)}

    def exact(Ca):
        r = lambda t: 1.0 + sum(Ca * F1[n] * eval_legendre(n, t) for n in F1) \
            + sum(Ca * Ca * F2[n] * eval_legendre(n, t) for n in F2)
        a, b = r(1.0), r(0.0)
        return (a - b) / (a + b)

    errs = [abs(exact(c) - spt.deformation(F1, F2, c)) for c in (1e-2, 5e-3)]
    assert errs[0] < 5e-5 and 6.0 < errs[0] / errs[1] < 10.0      # third order: halving Ca gives 1/8
    assert abs(exact(1e-2) - spt.deformation(F1, None, 1e-2)) > 1e-5   # the second-order part matters


def test_surfactant_quadrupole_theory_reproduces_table2():
    """Table 2 lists, for the same numerical D, its relative difference to the first- and second-order
    values; with differences taken relative to the numerical value, D2 / D1 = (1 - e2) / (1 - e1). The
    oracle's first-order (Mandal et al.) and second-order (Appendix A.1, s = 2, beta_t = 1) coefficients
    reproduce that ratio to 1e-6 at all three capillary numbers (the table's 5 digits allow about 1e-6)."""
    for drop, ca, e1, e2 in table2():
        if drop != "surfactant":
            continue
        D1 = spt.quad_D(2.0, 0.01, ca, clean=False, bt=1.0, order=1)
        D2 = spt.quad_D(2.0, 0.01, ca, clean=False, bt=1.0, order=2)
        assert abs(D2 / D1 - (1.0 - e2) / (1.0 - e1)) < 1e-6, (ca, D2 / D1)
        assert D1 < D2                                       # the numerical D lies above both


def test_first_order_theories_agree_with_the_uniform_closed_forms():
    """Eq. DS2 and Eq. DS2clean to first order are 3/4 F_20^(1) of the matching first-order shape
    (Nganguia et al., Taylor)."""
    for R, Q in ((0.1, 1.0), (2.0, 0.5), (6.0, 2.0)):
        for clean in (True, False):
            Ca = 1e-6
            D1 = spt.deformation(spt.uniform_first(R, Q, clean), None, Ca)
            assert abs(D1 - spt.uniform_D_closed(R, Q, Ca, clean)) < 1e-5 * abs(D1)   # its Ca^2 part: ~1e-6
