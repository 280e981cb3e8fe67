"""Host-side helpers of the learned starting bound (no GPU): seeded initial
weights, epoch orders, and the offset rule that turns network outputs into
proposed bounds by the expected number of decide runs."""
import math

import numpy as np

from paper_1709_09990_gb300 import learned


def test_initial_weights_are_seeded_and_bounded():
    a = learned.init_params(7)
    b = learned.init_params(7)
    c = learned.init_params(8)
    assert a.dtype == np.float32 and a.shape == (learned.N_PARAMS,)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    w1, b1 = a[:32 * 12], a[32 * 12: 32 * 12 + 32]
    w2, b2 = a[32 * 12 + 32: 32 * 12 + 64], a[32 * 12 + 64:]
    assert np.all(np.abs(w1) <= 1 / math.sqrt(12)) and np.all(np.abs(w2) <= 1 / math.sqrt(32))
    assert not b1.any() and not b2.any()
    assert np.abs(w1).max() > 0.5 / math.sqrt(12)  # spread over the range, not collapsed


def test_epoch_orders_are_permutations():
    p = learned.epoch_orders(50, 4, 3)
    assert p.shape == (4, 50) and p.dtype == np.int32
    for row in p:
        assert sorted(row.tolist()) == list(range(50))
    assert not np.array_equal(p[0], p[1])
    assert np.array_equal(p, learned.epoch_orders(50, 4, 3))


def test_offset_rule_on_hand_worked_cases():
    # one graph, tw = 5, lower bound 3, exact prediction 5.0.  Proposal
    # k0 = max(rint(5 + off), 3) costs tw - k0 + 1 runs below tw (no runs up to
    # tw - 1, then the yes) and k0 - tw + 1 runs from above (+1 for the no at
    # tw - 1 when tw > lb), plus 0.25 when k0 > tw:
    #   off -2 -> k0 3: 3;  -1.5 -> 4: 2;  -1 -> 4: 2;  -0.5 -> 4: 2;
    #   0 -> 5: 1 + 1 = 2;  0.5 -> 6: 2 + 1 + 0.25 = 3.25
    # the first of the cheapest offsets wins
    assert learned.choose_offset(np.array([5.0]), np.array([5]), np.array([3])) == -1.5
    # tw at the lower bound: a proposal at tw needs no certifying "no" run,
    # one below it is clamped to the bound, so every offset up to 0 costs one
    # run and the first one is kept
    assert learned.choose_offset(np.array([5.0]), np.array([5]), np.array([5])) == -2.0
    # predictions one above tw: offset -1 brings them onto tw
    pred = np.array([8.0, 9.0, 10.0])
    tw = np.array([7, 8, 9])
    lb = np.array([2, 2, 2])
    assert learned.choose_offset(pred, tw, lb) in (-2.0, -1.5, -1.0)
    k0 = np.maximum(np.rint(pred + learned.choose_offset(pred, tw, lb)), lb)
    assert np.all(k0 <= tw)
