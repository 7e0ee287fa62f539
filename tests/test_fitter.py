"""The library's relaxation fitter (fw2_fit_relaxation, Sec. 4.1), a host
computation: its model curves equal the oracle's independent evaluation of
Eq. (dispersion_relations), its grid search equals the oracle's restatement
of the paper's coarse-to-fine search, and the paper's search with the polish
meets the paper's accuracy claims for Table 2's target."""
import math

import numpy as np
import pytest

import synth
from oracle import analytic as an
from oracle import fit_relaxation as fr
from paper_2106_11476_gb300 import fw2


def _params(rng, N):
    return {"kappa1": rng.uniform(0.8, 1.2), "kappa2": rng.uniform(0.8, 1.2),
            "d1": list(10 ** rng.uniform(2, 9, N)), "alpha1": list(10 ** rng.uniform(5, 11, N)),
            "d2": list(10 ** rng.uniform(2, 9, N)), "alpha2": list(10 ** rng.uniform(5, 11, N))}


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_curves_equal_the_oracle_dispersion_relation(fw2lib, N):
    rng = np.random.default_rng(N)
    f = np.linspace(0.5e6, 25e6, 101)
    for _ in range(5):
        p = _params(rng, N)
        att, c = fw2.fw2_relaxation_curves(p, 1540.0, f)
        att_o, c_o = an.model_curves(f, 1540.0, p)
        np.testing.assert_allclose(att, att_o, rtol=1e-11)
        np.testing.assert_allclose(c, c_o, rtol=1e-12)


def _table2_cost(f_ref):
    f = np.linspace(1e6, 20e6, 77)
    att, c = an.model_curves(f, 1540.0, synth.TABLE2)
    return (fr.W_ALPHA * fr.nmse(att, an.power_law_db_cm(f, 0.5, 1.0))
            + (1 - fr.W_ALPHA) * fr.nmse(c, an.kk_phase_velocity(f, 0.5, 1.0, 1540.0, f_ref)))


def test_grid_search_equals_the_oracle_search(fw2lib):
    """3 values per dimension, two finer searches, N = 2: the library's grid
    reaches the cost the oracle's restatement of the search reaches."""
    f_ref = 10.5e6
    lib = fw2.fw2_fit_relaxation(0.5, 1.0, 2, grid_points=3, refinements=2, polish_iterations=0, f_ref=f_ref)
    orc = fr.fit_grid(0.5, 1.0, 2, f_ref=f_ref, points=3, refinements=2)
    assert lib["evaluations"] == 3 * 3 ** 10
    assert abs(lib["J"] - orc["J"]) <= 1e-10 * orc["J"], (lib["J"], orc["J"])


def test_paper_search_meets_the_paper_claims_for_table2(fw2lib):
    """Table 2's target (alpha0 = 0.5 dB/cm/MHz, y = 1, N = 2) with the
    paper's search (5 values per dimension over Table 2's bounds, four finer
    searches each 30 % narrower): the grid alone reaches a lower cost than
    Table 2's own values under the same cost (c0 at the band centre), and the
    polish that follows meets the paper's claims, under 5 % attenuation error
    from 2 to 20 MHz and under 0.5 % phase-velocity error."""
    p = fw2.fw2_fit_relaxation(0.5, 1.0, 2)
    assert p["f_ref"] == 10.5e6
    assert p["evaluations"] >= 5 * 5 ** 10
    assert p["J_grid"] <= _table2_cost(10.5e6)
    assert p["J"] <= p["J_grid"]
    assert p["max_att_rel_err_2_20MHz"] < 0.05 and p["max_phase_rel_err"] < 0.005
    # the reported errors are those of the returned set
    f = np.linspace(1e6, 20e6, 77)
    att, c = an.model_curves(f, 1540.0, p)
    err = np.max(np.abs(att / an.power_law_db_cm(f, 0.5, 1.0) - 1)[f >= 2e6])
    assert abs(err - p["max_att_rel_err_2_20MHz"]) < 1e-9
    for key in ("d1", "d2"):
        assert all(1e2 <= v <= 1e10 for v in p[key])
    for key in ("alpha1", "alpha2"):
        assert all(1e5 <= v <= 1e12 for v in p[key])


def test_table2_cost_depends_on_the_reference_frequency():
    """Reading R1: the phase-velocity target is anchored at c0 at f_ref, which
    the paper does not state; with f_ref at the band centre Table 2 scores
    J = 0.025, with 3 MHz 2.2 (its 0.12 % offset there is large against the
    target's variance)."""
    assert _table2_cost(10.5e6) < 0.03
    assert _table2_cost(3e6) > 2.0


@pytest.mark.parametrize("patch", [{"n_relax": 0}, {"n_relax": 5}, {"alpha0": -1.0}, {"f_hi": 0.5e6},
                                   {"shrink": 1.0}, {"grid_points": 9, "n_relax": 4}])
def test_fit_rejects_bad_requests(fw2lib, patch):
    args = {"alpha0": 0.5, "y": 1.0, "n_relax": 2}
    args.update(patch)
    a0, y, N = args.pop("alpha0"), args.pop("y"), args.pop("n_relax")
    with pytest.raises(fw2.Fw2Error):
        fw2.fw2_fit_relaxation(a0, y, N, **args)
