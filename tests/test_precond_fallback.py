"""The learned preconditioner's fallback rule (paper_2405_01522_gb300.precond.should_fall_back),
host logic only: a learned run drops its network when none of the last `patience`
energies sets a new minimum by more than the tolerance."""
from paper_2405_01522_gb300.precond import should_fall_back


def test_steady_descent_keeps_the_network():
    trace = [-1.0 - 0.1 * k for k in range(20)]
    assert not any(should_fall_back(trace[:i], 3, 1e-6) for i in range(len(trace) + 1))


def test_stagnation_or_rise_for_patience_steps_falls_back():
    trace = [-1.0, -1.5, -1.7, -1.69, -1.6999, -1.68]
    assert should_fall_back(trace, 3, 1e-6)          # three steps without a new minimum
    assert not should_fall_back(trace, 4, 1e-6)      # -1.7 itself was a new minimum
    assert not should_fall_back(trace[:5], 3, 1e-6)  # only two steps since the minimum


def test_gains_below_the_tolerance_count_as_stagnation():
    trace = [-2.0, -2.0 - 1e-9, -2.0 - 2e-9, -2.0 - 3e-9]
    assert should_fall_back(trace, 3, 1e-6)
    assert not should_fall_back(trace, 3, 1e-10)


def test_short_histories_and_disabled_rule():
    assert not should_fall_back([], 1, 1e-6)
    assert not should_fall_back([-1.0], 1, 1e-6)
    assert not should_fall_back([-1.0, 0.0, 1.0], 0, 1e-6)
