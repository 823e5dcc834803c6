"""The oracle's constants against the numbers the paper prints
(tests/golden/paper_constants.json, each entry with its citation)."""
import json
import os
from fractions import Fraction

import oracle
from oracle import brute, nms

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def test_kdm_value():
    assert brute.K_DM == Fraction(GOLD["K_DM"]["value"]).limit_denominator(1000)
    # the C oracle uses the same constant: delay of 1 DM, 1 MHz vs f_ref -> K*(1 - 1/fr^2)/tsamp
    D = oracle.delay_table(1, 0.5, 1.5, 1.0, [1.0])   # one channel centred at 1.0 MHz, f_ref = 1.5
    assert D[0, 0] == round(GOLD["K_DM"]["value"] * (1.0 - 1.0 / 2.25))


def test_matching_tolerances():
    assert nms.DM_TOL == GOLD["tp_dm_tolerance"]["value"]
    assert nms.TOA_TOL == GOLD["tp_toa_tolerance"]["value"]
