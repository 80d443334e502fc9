"""Partitioning efficiency model (Sec. 3.4): the oracle against the paper's
worked example and invariants, the C-ABI library against the oracle."""
import json
import os

import pytest

from oracle import partition
from oracle.mesh import Forest, build_forest
from paper_1904_03317_gb300 import gmg as G
from paper_1904_03317_gb300 import inputs
from tests.helpers import small_workloads

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")))
EXAMPLE = GOLDEN["partition_example"]["value"]
UNIT_SQUARE = inputs.CoarseMesh(2, (1, 1, 1), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1904_03317_gb300 import build
    build.build()


def example_forest():
    f = Forest(UNIT_SQUARE)
    f._refine_cell(0, (0, 0, 0))
    f._refine_cell(1, (0, 0, 0))  # the first (bottom-left) child
    assert f.is_balanced()
    return f


def example_mesh():
    m = G.Mesh(UNIT_SQUARE)
    m.refine([1])
    m.refine([1, 0, 0, 0])  # leaves in z-order: the first child comes first
    return m


def test_oracle_reproduces_paper_example():
    r = partition.model(example_forest(), EXAMPLE["n_parts"])
    assert r["n_cells"] == EXAMPLE["n_cells"]
    assert r["w_opt"] == EXAMPLE["w_opt"]
    assert r["w_sync"] == EXAMPLE["w_sync"]
    assert r["w"] == EXAMPLE["w"]
    assert r["efficiency"] == EXAMPLE["efficiency"]


def test_oracle_first_child_rule_on_example():
    own = partition.owners(example_forest(), 3)
    # the root and the refined child follow the first leaf (part 0)
    assert own[0][(0, 0, 0)] == 0 and own[1][(0, 0, 0)] == 0
    # every part owns some leaf
    assert sorted(set(own[2].values()) | {own[1][c] for c in own[1] if c != (0, 0, 0)}) == [0, 1, 2]


@pytest.mark.parametrize("name", ["2d_q1_circle", "3d_q1_sphere"])
def test_oracle_invariants(name):
    w = small_workloads()[name]
    f = build_forest(w.coarse, w.rounds)
    total = sum(len(c) for c in f.cells)
    one = partition.model(f, 1)
    assert one["efficiency"] == 1.0 and one["w"] == total
    for n in (2, 3, 16, 1000, 10 ** 6):
        r = partition.model(f, n)
        assert r["w_opt"] <= r["w_sync"] <= r["w"] <= total
        assert 0 < r["efficiency"] <= 1
        assert all(1 <= wl <= nl for wl, nl in zip(r["w_level"], r["n_cells"]))


def test_library_reproduces_paper_example():
    r = example_mesh().partition_model(EXAMPLE["n_parts"])
    assert r["n_cells"] == EXAMPLE["n_cells"]
    assert (r["w_opt"], r["w_sync"], r["w"], r["efficiency"]) == (
        EXAMPLE["w_opt"], EXAMPLE["w_sync"], EXAMPLE["w"], EXAMPLE["efficiency"])


@pytest.mark.parametrize("name", list(small_workloads()))
def test_library_matches_oracle(name):
    w = small_workloads()[name]
    f = build_forest(w.coarse, w.rounds)
    m = G.build_mesh(w)
    for n in (1, 2, 5, 64, 5000, 10 ** 7):
        a, b = m.partition_model(n), partition.model(f, n)
        assert a["n_cells"] == b["n_cells"] and a["w_level"] == b["w_level"]
        assert a["w_sync"] == b["w_sync"] and a["w"] == b["w"]
        assert a["w_opt"] == pytest.approx(b["w_opt"], rel=1e-15)


def test_library_rejects_bad_parts():
    m = example_mesh()
    with pytest.raises(Exception):
        m.partition_model(0)
