"""Host rule for the stream pipeline's adjoint tape (no GPU): the whole run
is kept as one segment when its tape fits the budget, otherwise the run is
cut into segments of about sqrt(n_steps) steps that the sweep recomputes."""
import math

from paper_2511_22468_gb300.stream import TAPE_BUDGET, tape_interval


def test_whole_run_kept_when_it_fits():
    # the stream workload: N = 1e4 (10240 padded), 6000 steps -> 4.4 GB
    assert 72.0 * 10240 * 6000 <= TAPE_BUDGET
    assert tape_interval(10_000, 6000) == 6000
    assert tape_interval(10_000, 1) == 1


def test_segments_when_the_tape_is_too_large():
    n, steps = 1_000_000, 6000          # 72 B x 1000448 x 6000 = 432 GB
    assert tape_interval(n, steps) == round(math.sqrt(steps))
    # the budget is honoured at the boundary
    npad = 10240
    exact = int(TAPE_BUDGET // (72 * npad))
    assert tape_interval(10_000, exact) == exact
    assert tape_interval(10_000, exact + 1) == round(math.sqrt(exact + 1))
