"""The learning-rate modulation of the paper's offline training (Sec. 5.3,
eq. learning_rate_modulation): host logic, no GPU."""
import math

from paper_2109_14403_gb300.linear import lr_schedule


def test_modulation_endpoints_period_and_decay():
    a_min, a_max, M, g = 1.5e-3, 1.5e-2, 50, 0.999
    assert math.isclose(lr_schedule(0), a_max)
    # a minimum after M epochs, back to the (decayed) maximum after 2M: period 2M
    assert math.isclose(lr_schedule(M), g ** M * a_min)
    assert math.isclose(lr_schedule(2 * M), g ** (2 * M) * a_max)
    assert math.isclose(lr_schedule(M // 2), g ** (M // 2) * 0.5 * (a_min + a_max))
    # never below the decayed minimum
    assert all(lr_schedule(m) >= g ** m * a_min * (1 - 1e-12) for m in range(300))
