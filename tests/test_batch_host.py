"""Host logic of the batch autotuner (no GPU): problem classes, the tuned
tile lookup and the record."""
from paper_1904_03317_gb300 import batch


def test_problem_class_is_half_decades_of_the_leaf_count():
    assert batch.problem_class(3, 2, 1) == (3, 2, 0)
    assert batch.problem_class(3, 2, 3) == (3, 2, 0)      # 2 log10(3) = 0.95
    assert batch.problem_class(3, 2, 4) == (3, 2, 1)      # 1.20
    assert batch.problem_class(2, 1, 10 ** 4) == (2, 1, 8)
    assert batch.problem_class(2, 1, 31622) == (2, 1, 8)  # just below 10^4.5
    assert batch.problem_class(2, 1, 31623) == (2, 1, 9)
    assert batch.problem_class(3, 1, 0) == (3, 1, 0)


def test_tile_lookup_and_record():
    t = batch.Tuning()
    t.tile[(3, 2, 8)] = 2
    t.tile_ms[(3, 2, 8)] = {2: 1.25, 4: 1.5, 8: 2.0}
    t.streams, t.streams_ms = 32, {8: 10.0, 32: 7.5}
    assert batch.tile_for(t, 3, 2, 12000) == 2      # class (3, 2, 8)
    assert batch.tile_for(t, 3, 2, 50000) == 0      # untuned class: library default
    assert batch.tile_for(t, 2, 2, 12000) == 0      # 2D: no bricks
    r = t.record()
    assert r["tile_brick_min_members"] == {"3d_q2_leaves_1e4": 2}
    assert r["tile_ms_per_solve"]["3d_q2_leaves_1e4"] == {"2": 1.25, "4": 1.5, "8": 2.0}
    assert r["streams"] == 32 and r["streams_ms_per_batch"] == {"8": 10.0, "32": 7.5}


class _FakeMesh:
    def __init__(self, n):
        self.n = n

    def num_leaves(self):
        return self.n


class _W:
    def __init__(self, dim, degree):
        self.coarse = type("C", (), {"dim": dim})()
        self.degree = degree


def test_class_counts():
    ws = [_W(3, 2), _W(3, 2), _W(2, 1), _W(3, 1)]
    ms = [_FakeMesh(1000), _FakeMesh(2000), _FakeMesh(1000), _FakeMesh(1000)]
    assert batch.class_counts(ws, ms) == {(3, 2, 6): 2, (2, 1, 6): 1, (3, 1, 6): 1}
