"""The checkpoint-interval policy of recorded rollouts (host only): the
interval that fits the memory budget and recomputes least."""
from paper_2510_17335_gb300 import mpm


def _recomputed(S, K):
    return S - (S - K * (-(-S // K) - 1))


def test_best_interval_recomputes_least():
    # 500 substeps with room for at most 70 per segment: 63 leaves a last
    # segment of 59 (441 recomputed), 70 would leave 10 (490 recomputed)
    assert mpm.best_interval(500, 70) == 63
    # the whole 2,000-substep rollout with room for 550: 500 (1,500 recomputed, not 1,650)
    assert mpm.best_interval(2000, 550) == 500
    assert mpm.best_interval(100, 100) == 100 and mpm.best_interval(100, 1) == 1
    # brute force: no interval that fits recomputes less
    for S in (7, 100, 333):
        for k_max in (1, 5, 40, S):
            K = mpm.best_interval(S, k_max)
            assert K <= k_max and all(_recomputed(S, K) <= _recomputed(S, k) for k in range(1, k_max + 1))


def test_checkpoint_interval_fits_the_budget():
    n, nodes = 1 << 20, 128 ** 3
    state, sub = mpm.record_bytes(n, nodes)
    for S, free in ((2000, 270 << 30), (2000, 100 << 30), (100, 270 << 30), (500, 20 << 30)):
        reserve = max(8 << 30, free // 16)
        K = mpm.checkpoint_interval(S, n, nodes, free)
        used = (K + 1) * state + K * sub + (-(-S // K)) * state
        assert used <= free - reserve
        # no interval that fits recomputes less
        for k in range(1, S + 1):
            if (k + 1) * state + k * sub + (-(-S // k)) * state <= free - reserve:
                assert _recomputed(S, K) <= _recomputed(S, k)
    # the 1M bed's whole 2,000-substep rollout on a GB300 (about 270 GB free):
    # two segments of 1,000, half the rollout recomputed
    assert mpm.checkpoint_interval(2000, n, nodes, 270 << 30) == 1000
    # a 100-substep window fits whole: nothing recomputed
    assert mpm.checkpoint_interval(100, n, nodes, 270 << 30) == 100
    # no room for even one substep: K = 1
    assert mpm.checkpoint_interval(10, n, nodes, 8 << 30) == 1
