"""Host-side checks of program-structure tables (the ones hpa_load_structure
applies before it copies anything to the device), run through the C ABI on
the CPU: a valid binary passes, and each malformed table is refused with
HPA_E_INVALID_TABLE (or HPA_E_INVALID_ARG for a missing table)."""
import copy

import numpy as np
import pytest

import synth

NP = synth.NO_PARENT


@pytest.fixture(scope="module")
def hpa_mod():
    from paper_2109_06931_gb300 import hpa
    return hpa


@pytest.fixture(scope="module")
def plain():
    return synth.PLAIN.binary()


def mutated(b, **changes):
    c = copy.copy(b)
    for k, v in changes.items():
        setattr(c, k, v)
    return c


def test_valid_binaries_pass(hpa_mod, plain):
    assert hpa_mod.validate_structure(plain) == (hpa_mod.HPA_OK, "")
    B = synth.make_binary(77, 300, 300 * 13_422, 15_000, 900, n_scc=3)
    assert hpa_mod.validate_structure(B)[0] == hpa_mod.HPA_OK


def bad(hpa_mod, b, status, words):
    st, msg = hpa_mod.validate_structure(b)
    assert st == status, (st, msg)
    assert words in msg, msg


def test_empty_and_overlapping_ranges(hpa_mod, plain):
    hi = plain.range_hi.copy()
    hi[5] = plain.range_lo[5]
    bad(hpa_mod, mutated(plain, range_hi=hi), hpa_mod.HPA_E_INVALID_TABLE, "empty")
    lo = plain.range_lo.copy()
    lo[7] = plain.range_hi[6] - np.uint64(1)
    bad(hpa_mod, mutated(plain, range_lo=lo), hpa_mod.HPA_E_INVALID_TABLE, "overlaps")
    perm = np.arange(plain.range_lo.shape[0])
    perm[[10, 11]] = perm[[11, 10]]
    bad(hpa_mod, mutated(plain, range_lo=plain.range_lo[perm], range_hi=plain.range_hi[perm],
                         range_node=plain.range_node[perm]), hpa_mod.HPA_E_INVALID_TABLE, "out of order")


def test_range_node_and_span(hpa_mod, plain):
    nd = plain.range_node.copy()
    nd[3] = plain.node_parent.shape[0]
    bad(hpa_mod, mutated(plain, range_node=nd), hpa_mod.HPA_E_INVALID_TABLE, "names node")
    lo, hi = plain.range_lo.copy(), plain.range_hi.copy()
    lo[-1] = lo[0] + np.uint64(1 << 32)
    hi[-1] = lo[-1] + np.uint64(16)
    bad(hpa_mod, mutated(plain, range_lo=lo, range_hi=hi), hpa_mod.HPA_E_INVALID_TABLE, "span")


def test_tree_rules(hpa_mod, plain):
    kind = plain.node_kind
    funcs = np.nonzero(plain.node_parent == NP)[0]
    inner = np.nonzero(plain.node_parent != NP)[0]
    # a FUNC node given a parent
    par = plain.node_parent.copy()
    par[funcs[1]] = inner[0]
    bad(hpa_mod, mutated(plain, node_parent=par), hpa_mod.HPA_E_INVALID_TABLE, "roots")
    # a parent in another function
    v = next(int(x) for x in inner if plain.node_func[x] != plain.node_func[funcs[0]])
    par = plain.node_parent.copy()
    par[v] = funcs[0]
    bad(hpa_mod, mutated(plain, node_parent=par), hpa_mod.HPA_E_INVALID_TABLE, "different functions")
    # two non-FUNC nodes of one function that are each other's parent
    f = plain.node_func[inner[0]]
    a, b = (int(x) for x in inner[plain.node_func[inner] == f][:2])
    par = plain.node_parent.copy()
    par[a], par[b] = b, a
    bad(hpa_mod, mutated(plain, node_parent=par), hpa_mod.HPA_E_INVALID_TABLE, "cycle")
    # two FUNC nodes for one function
    fn = plain.node_func.copy()
    fn[funcs[1]] = fn[funcs[0]]
    fn[plain.node_func == plain.node_func[funcs[1]]] = fn[funcs[0]]
    bad(hpa_mod, mutated(plain, node_func=fn), hpa_mod.HPA_E_INVALID_TABLE, "two FUNC nodes")
    # an unknown kind
    k = kind.copy()
    k[inner[0]] = 9
    bad(hpa_mod, mutated(plain, node_kind=k), hpa_mod.HPA_E_INVALID_TABLE, "kind")


def test_call_site_rules(hpa_mod, plain):
    ce = plain.cs_callee.copy()
    ce[0] = plain.n_funcs
    bad(hpa_mod, mutated(plain, cs_callee=ce), hpa_mod.HPA_E_INVALID_TABLE, "n_funcs")
    # the call site's node is a LINE node of the caller, not its CALL node
    cn = plain.cs_node.copy()
    cn[0] = plain.node_parent[plain.cs_node[0]]
    bad(hpa_mod, mutated(plain, cs_node=cn), hpa_mod.HPA_E_INVALID_TABLE, "CALL node")
    # the CALL node of another function
    other = next(e for e in range(1, len(cn)) if plain.cs_caller[e] != plain.cs_caller[0])
    cn = plain.cs_node.copy()
    cn[0] = plain.cs_node[other]
    bad(hpa_mod, mutated(plain, cs_node=cn), hpa_mod.HPA_E_INVALID_TABLE, "CALL node")


def test_missing_tables(hpa_mod, plain):
    empty = mutated(plain, range_lo=np.zeros(0, np.uint64), range_hi=np.zeros(0, np.uint64),
                    range_node=np.zeros(0, np.uint32))
    bad(hpa_mod, empty, hpa_mod.HPA_E_INVALID_ARG, "range")
