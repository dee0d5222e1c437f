"""The convergence bookkeeping of the bench and of the warm-start evaluation (CPU).

Sect. 2.4, Eqs. 4-6: Q_99 is the 99th percentile of the ratio change of the cell temperatures
between consecutive iterations, and Delta = max(Q_prev / Q, Q / Q_prev).  The literal criterion
asks Q_99 < 1.02; the Delta test asks Q_99 < 2 and Delta < 1.02.  The histories below are
hand-made (the first is the shape the 256^3 cloud shows), so that the iteration each criterion
picks, and the time summed up to it, can be read off by eye."""
import bench
from paper_1112_1071_gb300 import learned

CLOUD = [5.8768, 1.18767, 1.16492, 1.16485, 1.165]      # falls to its Monte-Carlo floor
FALLING = [4.0, 1.5, 1.1, 1.019, 1.015]                # reaches 1.02 at the 4th iteration
MS = [10.0, 20.0, 30.0, 40.0, 50.0]


def test_literal_criterion_needs_the_quantile_below_1_02():
    assert bench.converged_at(CLOUD, MS, 1.02) == (None, None)
    assert bench.converged_at(FALLING, MS, 1.02) == (4, 100.0)
    assert learned.converged_at(CLOUD, 1.02) is None
    assert learned.converged_at(FALLING, 1.02) == 4


def test_delta_test_needs_a_settled_quantile_below_2():
    # Delta(1.18767, 1.16492) = 1.0195 < 1.02 with Q < 2: the 3rd iteration, after 60 ms
    assert bench.converged_at(CLOUD, MS, 2.0, 1.02) == (3, 60.0)
    assert learned.converged_at(CLOUD, 2.0, 1.02) == 3
    # Q below 2 from the 2nd iteration, but Delta(4.0, 1.5) and Delta(1.5, 1.1) are large and
    # Delta(1.1, 1.019) = 1.079: not before the 5th (Delta(1.019, 1.015) = 1.004)
    assert bench.converged_at(FALLING, MS, 2.0, 1.02) == (5, 150.0)
    assert learned.converged_at(FALLING, 2.0, 1.02) == 5
    # a history that stays above 2 never passes, however settled
    assert bench.converged_at([3.0, 3.0, 3.0], MS[:3], 2.0, 1.02) == (None, None)


def test_first_iteration_is_never_converged_in_the_bench():
    # the first quantile compares with the starting temperatures (10 K): the bench counts from
    # the 2nd iteration even under the literal criterion
    assert bench.converged_at([1.0, 1.5, 1.01], [1.0, 1.0, 1.0], 1.02) == (3, 3.0)


def test_convergence_fields_take_the_median_over_steps():
    steps = [[{"Q": q, "ms_total": m} for q, m in zip(CLOUD, MS)],
             [{"Q": q, "ms_total": 2 * m} for q, m in zip(CLOUD, MS)],
             [{"Q": q, "ms_total": 3 * m} for q, m in zip(FALLING, MS)]]
    f = bench.convergence_fields(steps, 5)
    assert f["iterations_to_converged_delta"] == 3                   # median of 3, 3, 5
    assert f["time_to_converged_delta_ms"] == 120.0                  # median of 60, 120, 450
    assert f["iterations_to_converged"] == 4                         # only the third step converges
    assert f["time_to_converged_ms"] == 300.0
    assert f["q99_history"] == [round(q, 5) for q in FALLING]
