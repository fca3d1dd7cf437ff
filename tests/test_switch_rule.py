"""The mixed form's FP32 -> FP64 switch rule (reading R22), replayed on the host through the
library (lobpcg_mixed_switch_replay, the code the solver runs), on residual histories
whose answer is worked out by hand."""
import numpy as np
import pytest

import paper_2305_06668_gb300 as lb


def replay(rk, tol=0.0):
    return lb.mixed_switch_replay(np.asarray(rk, dtype=np.float64), tol)


def test_loss_of_a_fast_rate_leaves_at_the_second_slow_iteration():
    """r_i = 0.3^i for i = 0..7, then flat at r_7 (the FP32 floor).  At i = 8 the first slow
    step (r_8 = r_7) is one slow iteration; at i = 9 the second: fast over i-5..i-2 =
    4..7 (factor 0.027 <= 0.216) and r_9 <= 1e-2 r_0, so the rule leaves after i = 9."""
    r = [0.3 ** i for i in range(8)] + [0.3 ** 7] * 6
    assert replay(r) == 9


def test_one_slow_iteration_does_not_leave():
    """A single slow step between fast ones is not a loss of rate: 0.3^i with r_8 = r_7 and
    then the fast decay resumes; with a plateau of 1 the fast rule never fires, and the
    10% rule needs 2 iterations without improvement."""
    r = [0.3 ** i for i in range(8)] + [0.3 ** 7] + [0.3 ** (7 + j) for j in range(1, 6)]
    assert replay(r) == -1


def test_no_ten_percent_gain_for_five_iterations_at_any_level():
    """r_i = 0.99^i never falls below 1% of r_0 in 8 steps, is never fast, and improves by
    10% on its best (r_0) only at i = 11: the count of non-improving iterations reaches 5 at
    i = 5."""
    r = [0.99 ** i for i in range(8)]
    assert replay(r) == 5


def test_two_iterations_without_gain_once_below_one_percent():
    """Slow decay 0.85 per step to below 1% of r_0 (never fast: 0.85^3 = 0.61 > 0.216), then
    flat.  Below 1%, two iterations without a 10% gain suffice."""
    r = [0.85 ** i for i in range(40)]
    first_below = int(np.argmax(np.array(r) <= 1e-2))
    r = r[: first_below + 1] + [r[first_below]] * 5
    # the best is set at first_below (a >10% gain); the flat steps at first_below+1, +2 count 1, 2
    assert replay(r) == first_below + 2


def test_fixed_threshold_leaves_at_the_first_residual_below_it():
    """switch_tol > 0 replaces the floor rules: the first i with r_i <= switch_tol."""
    r = [1.0, 0.5, 0.2, 0.05, 0.04, 0.01, 0.001]
    assert replay(r, tol=0.045) == 4
    assert replay(r, tol=1e-6) == -1
    # a plateau does not end the phase when a threshold is set
    assert replay([1.0] * 20, tol=1e-3) == -1


def test_empty_history_and_argument_errors():
    assert replay([]) == -1
    with pytest.raises(lb.LobpcgError) as e:
        replay([1.0], tol=-1.0)
    assert e.value.status == lb.EINVAL
