"""bingo_policy_make: walk policies from their real-valued parameters (host only, no GPU)."""
import pytest


@pytest.fixture(scope="module")
def B():
    from paper_2504_10233_gb300 import _build

    _build.build()
    import paper_2504_10233_gb300 as B

    B.load()
    return B


def test_node2vec_thresholds(B):
    # Eq. node2vec: f = 1/p, 1, 1/q at distance 0, 1, 2, accepted with f / max f
    assert list(B.policy(B.NODE2VEC, 80, n2v_pq=(2.0, 0.5)).n2v_accept) == [1 << 30, 1 << 31, 1 << 32]
    assert list(B.policy(B.NODE2VEC, 80, n2v_pq=(0.5, 2.0)).n2v_accept) == [1 << 32, 1 << 31, 1 << 30]
    assert list(B.policy(B.NODE2VEC, 80, n2v_pq=(1.0, 1.0)).n2v_accept) == [1 << 32] * 3
    p = B.policy(B.NODE2VEC, 80, n2v_pq=(3.0, 1.0))  # f = 1/3, 1, 1: a non-dyadic ratio rounds to the nearest step
    assert list(p.n2v_accept) == [round(2 ** 32 / 3), 1 << 32, 1 << 32]


def test_ppr_threshold(B):
    assert B.policy(B.PPR, 100, 0.15).ppr_stop_u32 == 644245094  # round(0.15 * 2^32)
    assert B.policy(B.PPR, 100, 0.0).ppr_stop_u32 == 0
    assert B.policy(B.PPR, 100, 1.0).ppr_stop_u32 == 0xFFFFFFFF
    assert B.policy(B.PPR, 100, 7).ppr_stop_u32 == 7  # an int is taken as the threshold itself


def test_invalid_parameters(B):
    for kw in ({"n2v_pq": (0.0, 1.0)}, {"n2v_pq": (1.0, float("inf"))}, {"n2v_pq": (-1.0, 1.0)}):
        with pytest.raises(B.BingoError):
            B.policy(B.NODE2VEC, 10, **kw)
    with pytest.raises(B.BingoError):
        B.policy(B.PPR, 10, 1.5)
    with pytest.raises(B.BingoError):
        B.policy(7, 10)
