"""Host logic of the serving summary: latency percentiles over every request
when some requests were still unfinished at the end of the window (their
latency is known only to be at least window end - arrival)."""
import numpy as np

from paper_1110_0899_gb300.serving import censored_latencies, censored_quantile


class _R:
    def __init__(self, arrival, finished):
        self.spec = {"arrival_s": arrival}
        self.finished_s = finished


def test_censored_quantile_exact_when_no_bound_reaches_it():
    vals = [(float(x), True) for x in range(1, 101)] + [(500.0, False)]
    v, exact = censored_quantile(vals, 0.5)
    assert v == 51.0 and exact          # the 51st of 101 is a finished request below the bound
    v, exact = censored_quantile(vals, 0.99)
    assert v == 100.0 and exact


def test_censored_quantile_is_a_lower_bound_past_the_censoring():
    vals = [(1.0, True), (2.0, True), (3.0, True), (4.0, False), (9.0, False)]
    v, exact = censored_quantile(vals, 0.99)
    assert v == 9.0 and not exact
    # a bound below a finished latency: the true order is unknown
    vals = [(1.0, True), (5.0, True), (2.0, False)]
    v, exact = censored_quantile(vals, 0.6)
    assert v == 2.0 and not exact
    assert censored_quantile([], 0.5) == (None, None)


def test_censored_latencies_counts_unfinished_requests():
    reqs = [_R(0.0, 1.5), _R(1.0, None), _R(2.0, 2.5), _R(40.0, None)]
    got = censored_latencies(reqs, wall=30.0)
    assert got == [(1.5, True), (29.0, False), (0.5, True), (0.0, False)]
    # with every request finished the quantile is the plain nearest-rank one
    lat = np.array([3.0, 1.0, 2.0, 5.0, 4.0])
    v, exact = censored_quantile([(x, True) for x in lat], 0.5)
    assert v == 3.0 and exact


def test_engine_choice_follows_the_measured_cost():
    from paper_1110_0899_gb300.serving import TEAM, TINY, choose_engine
    none = {TINY: None, TEAM: None}
    # above the tiny engine's limit, or with it off: the team engine
    assert choose_engine(2, 182, none, TEAM, 0) == TEAM
    assert choose_engine(3, 33, none, TEAM, 0) == TEAM
    assert choose_engine(2, 16, none, TEAM, 0, tiny=False) == TEAM
    # at most 64 words (2D L <= 32, 3D L <= 8): always the tiny engine
    assert choose_engine(2, 32, none, TEAM, 0) == TINY
    assert choose_engine(3, 8, {TINY: 9e9, TEAM: 1.0}, TINY, 100) == TINY
    # larger: team first, then tiny once, then the faster
    assert choose_engine(2, 64, none, TEAM, 1) == TEAM
    assert choose_engine(2, 64, {TINY: None, TEAM: 5000.0}, TEAM, 1) == TINY
    assert choose_engine(2, 64, {TINY: 800.0, TEAM: 5000.0}, TINY, 1) == TINY
    assert choose_engine(3, 32, {TINY: 20000.0, TEAM: 900.0}, TINY, 1) == TEAM
    # the other engine is timed again after reprobe_epochs on the same one
    assert choose_engine(2, 64, {TINY: 800.0, TEAM: 5000.0}, TINY, 7) == TINY
    assert choose_engine(2, 64, {TINY: 800.0, TEAM: 5000.0}, TINY, 8) == TEAM
    assert choose_engine(2, 64, {TINY: 800.0, TEAM: 5000.0}, TEAM, 1) == TINY


def test_tiny_split_of_the_batched_form():
    from paper_1110_0899_gb300.batched import tiny_split, tiny_words
    # words of the bit planes: (N / L) rows of ceil(L / 32) words
    assert tiny_words(2, 16) == 16 and tiny_words(2, 33) == 66 and tiny_words(2, 181) == 1086
    assert tiny_words(3, 8) == 64 and tiny_words(3, 32) == 1024
    specs = [dict(dim=2, L=32), dict(dim=2, L=33), dict(dim=3, L=8), dict(dim=3, L=9),
             dict(dim=2, L=181), dict(dim=2, L=182), dict(dim=3, L=32), dict(dim=3, L=33)]
    small, large, rest = tiny_split(specs, range(len(specs)))
    assert small == [0, 2]           # at most 64 words
    assert large == [1, 3, 4, 6]     # up to 32768 sites
    assert rest == [5, 7]            # beyond the tiny engine
