"""Pins of the oracle's group attributes (Sec. 2, Eqs. (csn_multi),
(egy_multi), (cse_multi); Verner fits, Eq. (PhI)) and of the frozen
constants the workloads carry."""
import json
import math
import os

import numpy as np
import pytest

from oracle import groups

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
GC = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "group_constants.json")))


def test_threshold_cross_sections():
    """Textbook threshold values: sigma_HI(13.6 eV) = 6.3e-18 cm^2 and the
    hydrogenic Z^-2 scaling for HeII, 6.3e-18/4; HeI 7.4e-18 (with the
    corrected epsilon_0 = 13.61 eV)."""
    assert groups.sigma("HI", 13.6) == pytest.approx(6.3e-18, rel=0.02)
    assert groups.sigma("HeII", 54.42) == pytest.approx(6.3e-18 / 4.0, rel=0.02)
    assert groups.sigma("HeI", 24.59) == pytest.approx(7.4e-18, rel=0.02)
    for sp, e in (("HI", 13.59), ("HeI", 24.58), ("HeII", 54.41)):
        assert groups.sigma(sp, e) == 0.0
    # far above threshold sigma falls roughly as eps^-3 for hydrogenic ions
    r = groups.sigma("HI", 400.0) / groups.sigma("HI", 200.0)
    assert 2 ** -3.5 < r < 2 ** -2.5


def test_one_band_matches_quoted_values():
    g = GOLD["groups_1e5K"]
    a = groups.group_attributes(groups.ONE_BAND, 1e5)
    assert a["sigN"][0, 0] == pytest.approx(g["one_band_sigN_HI"], rel=g["rtol"])
    assert a["egy"][0] / groups.EV == pytest.approx(g["one_band_egy_eV"], rel=g["rtol"])


def test_three_bands_consistency():
    a = groups.group_attributes(groups.THREE_BANDS, 1e5)
    one = groups.group_attributes(groups.ONE_BAND, 1e5)
    w = a["photon_fraction"]
    assert w.sum() == pytest.approx(1.0, rel=1e-10)
    # photon-weighted mean of the band cross sections / energies = one band
    assert np.dot(w, a["sigN"][:, 0]) == pytest.approx(one["sigN"][0, 0], rel=1e-8)
    assert np.dot(w, a["egy"]) == pytest.approx(one["egy"][0], rel=1e-8)
    # bands below a species' threshold have no cross section
    assert a["sigN"][0, 1] == 0 and a["sigN"][0, 2] == 0 and a["sigN"][1, 2] == 0
    for i, (lo, hi) in enumerate(groups.THREE_BANDS):
        e = a["egy"][i] / groups.EV
        assert lo < e < (hi if math.isfinite(hi) else 1e9)


def test_workload_literals_match_oracle():
    from paper_1304_7126_gb300 import workloads as W
    t = GC["three_band"]
    assert np.array_equal(np.array(W.BB3_SIGN), np.array(t["sigN"]))
    assert np.array_equal(np.array(W.BB3_SIGE), np.array(t["sigE"]))
    assert np.array_equal(np.array(W.BB3_EGY_EV), np.array(t["egy_eV"]))
    assert np.array_equal(np.array(W.BB3_PHOTON_FRACTION), np.array(t["photon_fraction"]))
    a = groups.group_attributes(groups.THREE_BANDS, 1e5)
    assert np.allclose(a["sigN"], t["sigN"], rtol=1e-12, atol=0)
    o = GC["one_band"]
    assert np.array_equal(np.array(W.BB1_SIGN), np.array(o["sigN"]))
    assert np.array_equal(np.array(W.BB1_SIGE), np.array(o["sigE"]))
    assert np.array_equal(np.array(W.BB1_EGY_EV), np.array(o["egy_eV"]))
