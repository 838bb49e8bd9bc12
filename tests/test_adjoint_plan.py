"""The checkpointed adjoint's recompute plan for one segment (lbm_adjoint_plan; host logic, no
GPU). For every segment length and number of free state buffers W, the schedule described in
include/lbm.h is walked step by step here: the states each reverse sweep needs are held when it
needs them, the buffers in use never exceed W, and the recompute count is 2 len - 2 - W (flat:
len - 1). Feasibility grows with W, and the smallest feasible W agrees with the memory limits the
GPU plan test relies on."""
import pytest


def _walk(length, W, starts):
    """Recompute steps and peak buffers of the schedule; asserts that every sweep finds its states."""
    m = len(starts) - 1
    if m == 0:
        return length - 1, length - 1
    s_m = starts[-1]
    L = length - s_m
    assert L >= 2  # the first pass alternates two of the last sub-segment's buffers
    kept = set(starts[1:-1])  # sub-segment starts held after the first pass
    last = {}                 # buffer slot of the last sub-segment -> state it holds
    recompute = 0
    # first pass: states 1 .. length - 1 once each; kept starts, the last sub-segment in place,
    # the others alternately in the last two slots (state s_m - 1 in slot L - 1)
    for i in range(1, length):
        recompute += 1
        if i in kept:
            continue
        slot = i - s_m if i >= s_m else L - 1 - ((s_m - 1 - i) & 1)
        last[slot] = i
    assert all(last[k] == s_m + k for k in range(L))  # the last sub-segment, swept first
    peak = len(kept) + L
    for j in range(m - 1, -1, -1):  # earlier sub-segments, latest first
        s_j, s_next = starts[j], starts[j + 1]
        assert s_j == 0 or s_j in kept
        assert s_next - s_j <= L + 1
        for i in range(s_j + 1, s_next):  # into the last sub-segment's buffers
            recompute += 1
            last[i - s_j - 1] = i
        assert all(last[i - s_j - 1] == i for i in range(s_j + 1, s_next))
    return recompute, peak


@pytest.fixture(scope="module")
def lbm():
    from paper_2605_27004_gb300 import build, lbm
    build.build()
    return lbm


def test_plans_fit_and_cost_as_stated(lbm):
    for length in range(1, 49):
        feasible = False
        for W in range(0, 50):
            starts = lbm.adjoint_plan(length, W)
            if length - 1 <= W:
                assert starts == [0], (length, W)
            if starts is None:
                assert not feasible, (length, W)  # feasibility grows with W
                continue
            feasible = True
            assert starts[0] == 0 and all(a < b for a, b in zip(starts, starts[1:])) and starts[-1] < length
            recompute, peak = _walk(length, W, starts)
            assert peak <= W, (length, W, starts)
            assert recompute == (length - 1 if len(starts) == 1 else 2 * length - 2 - W), (length, W, starts)


def test_smallest_plans(lbm):
    # K = 12 needs 5 working buffers (6 states with the restore target), K = 20 needs 7
    assert lbm.adjoint_plan(12, 4) is None and lbm.adjoint_plan(12, 5) is not None
    assert lbm.adjoint_plan(20, 6) is None and lbm.adjoint_plan(20, 7) is not None
    # the sub-segments the GPU plan test expects for K = 12 and 5 .. 8 working buffers
    assert lbm.adjoint_plan(12, 5) == [0, 4, 8]
    assert lbm.adjoint_plan(12, 6) == [0, 6]
    assert lbm.adjoint_plan(12, 7) == [0, 5]
    assert lbm.adjoint_plan(12, 8) == [0, 4]
    assert lbm.adjoint_plan(12, 11) == [0]


def test_plan_rejects_bad_arguments(lbm):
    with pytest.raises(lbm.LBMError):
        lbm.adjoint_plan(0, 3)
    with pytest.raises(lbm.LBMError):
        lbm.adjoint_plan(5, -1)
