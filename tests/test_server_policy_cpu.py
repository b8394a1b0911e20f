"""The request server's choice of launch shape (host rule, no GPU): first come,
first served between the shapes, the largest size class neutral between shapes 0
and 1, and the return to shape 0 once no request needs another shape.

Pool used throughout: class 0 a small size class (shape 0 only), class 1 the
largest size class (shapes 0 and 1), class 2 the large meshes (shape 1 only),
class 3 the huge meshes (shape 2 only)."""
import pytest

from paper_2103_16747_b300 import _lib as L

G3 = [[4, 1, 0, 0],     # shape 0: size classes
      [0, 1, 1, 0],     # shape 1: the largest class and the large-mesh group
      [0, 0, 0, 1]]     # shape 2: the huge-mesh group
G2 = [row[:3] for row in G3[:2]]


def pick(groups, cur, reqs):
    return L.fem_debug_pick_shape(groups, cur, reqs)


def test_one_shape_never_changes():
    assert pick([[2, 1]], 0, [(1, 0), (2, 1)]) == 0


def test_idle_server_stays_in_shape_0_and_returns_to_it():
    assert pick(G2, 0, []) == 0
    assert pick(G2, 1, []) == 0
    assert pick(G3, 2, []) == 0


def test_large_request_waits_for_older_small_ones_only():
    assert pick(G2, 0, [(5, 2)]) == 1                  # nothing of shape 0's own
    assert pick(G2, 0, [(3, 0), (5, 2)]) == 0          # an older small request runs first
    assert pick(G2, 0, [(7, 0), (5, 2)]) == 1          # the large one is older
    assert pick(G2, 0, [(3, 1), (5, 2)]) == 1          # the largest class runs in both shapes


def test_back_to_shape_0_by_age_or_when_large_work_is_done():
    assert pick(G2, 1, [(3, 1)]) == 0                  # only work shape 0 serves as well
    assert pick(G2, 1, [(4, 2), (9, 1)]) == 1          # a large request still unfinished
    assert pick(G2, 1, [(4, 2), (3, 0)]) == 0          # a small request older than it
    assert pick(G2, 1, [(2, 2), (3, 0)]) == 1          # a large request older than it


def test_three_shapes():
    # a huge request older than the live shape-1 work
    assert pick(G3, 1, [(2, 3), (5, 1)]) == 2
    # the largest class is not served by shape 2: an older request of it holds shape 1
    assert pick(G3, 1, [(6, 3), (5, 1)]) == 1
    # from shape 2 to the shape that serves the oldest waiting request
    assert pick(G3, 2, [(6, 3), (4, 0)]) == 0
    assert pick(G3, 2, [(6, 3), (4, 2)]) == 1
    assert pick(G3, 2, [(3, 3), (4, 0)]) == 2
    # the largest class waiting in shape 2 goes to shape 0 (the first shape serving it)
    assert pick(G3, 2, [(4, 1)]) == 0


def test_first_come_first_served_never_starves_a_class():
    # a stream of alternating arrivals: every change goes to the oldest waiting request
    reqs = [(1, 0), (2, 2), (3, 0), (4, 3), (5, 0)]
    cur, order = 0, []
    pending = list(reqs)
    while pending:
        cur = pick(G3, cur, pending)
        served = [r for r in pending if G3[cur][r[1]] > 0]
        assert served, "the chosen shape serves an unfinished request"
        done = min(served)
        order.append(done[0])
        pending.remove(done)
    assert order == [1, 2, 3, 4, 5]


@pytest.mark.parametrize("bad", [
    dict(groups=[[1, 0]], cur=0, reqs=[]),                       # class 1 served by no shape
    dict(groups=G2, cur=2, reqs=[]),                             # cur out of range
    dict(groups=G2, cur=0, reqs=[(1, 3)]),                       # class out of range
    dict(groups=[[1]] * 4, cur=0, reqs=[]),                      # four shapes
])
def test_arguments_are_checked(bad):
    with pytest.raises(L.FemError) as e:
        pick(bad["groups"], bad["cur"], bad["reqs"])
    assert e.value.code == L.FEM_ERR_ARG
