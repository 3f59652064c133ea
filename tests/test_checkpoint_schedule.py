"""Host logic of the binomial checkpoint replay (Sec. 3.2), simulated without a GPU."""
import pytest

from paper_2609_30039_gb300.adjoint import beta, repetitions, replay_stats, schedule, spine


def simulate(n, slots):
    acts = schedule(n, slots)
    state, slot, seen, done = 0, {}, [], False
    for a in acts:
        if a[0] == "save":
            assert a[1] < slots
            assert a[2] == state
            slot[a[1]] = state
        elif a[0] == "restore":
            state = slot[a[1]]
        elif a[0] == "advance":
            state += a[1]
            assert state <= n
        elif a[0] == "forward_done":
            assert state == n
            done = True
        elif a[0] == "adjoint":
            assert done and a[1] == state, (a, state)
            seen.append(a[1])
    assert seen == list(range(n - 1, -1, -1))
    return replay_stats(acts)


@pytest.mark.parametrize("n,slots", [(1, 1), (2, 1), (7, 2), (10, 3), (100, 5), (3000, 32), (4000, 16), (257, 4)])
def test_schedule_reverses_every_step_in_order(n, slots):
    st = simulate(n, slots)
    assert st["adjoint_steps"] == n
    if slots > 1:
        t = repetitions(n, slots - 1)
        # binomial bound: replay work is at most t forward steps per step, plus the first sweep
        assert st["forward_steps"] <= (t + 1) * n


def test_repetition_numbers_of_the_workloads():
    # r = min{r : C(c + r, r) >= n}
    assert repetitions(3000, 31) == 3 and beta(31, 3) == 5984 and beta(31, 2) == 528
    assert repetitions(4000, 15) == 5 and beta(15, 4) == 3876 < 4000 <= beta(15, 5)
    assert repetitions(4000, 31) == 3


def test_spine_is_increasing():
    sp = spine(3000, 31)
    assert sp == sorted(sp) and len(set(sp)) == len(sp) and sp[-1] < 3000


@pytest.mark.parametrize("n,slots", [(1, 1), (17, 3), (200, 8)])
def test_encoded_schedule_rows(n, slots):
    # the native executor's rows carry the same actions: one STOP after the forward sweep, one
    # transposed step per adjoint action, slots and step counts unchanged
    from paper_2609_30039_gb300 import fdtd as F
    from paper_2609_30039_gb300.adjoint import encode
    acts = schedule(n, slots)
    rows = encode(acts)
    assert rows.dtype.name == "int32" and rows.shape == (len(acts), 2)
    kinds = {"save": F.FDTD_ACT_SAVE, "restore": F.FDTD_ACT_RESTORE, "advance": F.FDTD_ACT_ADVANCE,
             "adjoint": F.FDTD_ACT_ADJOINT, "forward_done": F.FDTD_ACT_STOP}
    for a, r in zip(acts, rows):
        assert r[0] == kinds[a[0]]
        if a[0] in ("save", "restore", "advance"):
            assert r[1] == a[1]
        if a[0] == "adjoint":
            assert r[1] == 1
    assert int((rows[:, 0] == F.FDTD_ACT_STOP).sum()) == 1
    assert int((rows[:, 0] == F.FDTD_ACT_ADJOINT).sum()) == n
