"""C ABI checks that need no GPU: the library loads, exports every function include/hf.h
declares, and its host-side graph builder returns the documented status codes (Section III-A:
explicit edges, acyclic graphs) and the right topological levels."""
import ctypes
import os
import re

import networkx as nx
import numpy as np
import pytest

from paper_2203_08395_b300 import build as B
from paper_2203_08395_b300 import hf
from paper_2203_08395_b300 import synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    hf.load()


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:hf_status|void|const char\s*\*)\s+(hf_\w+)\s*\(", txt, flags=re.M)))


def test_every_declared_symbol_is_exported():
    names = _declared("hf.h")
    assert len(names) >= 27
    lib = ctypes.CDLL(hf.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_defaults_and_status_strings():
    o = hf.hf_run_opts_default()
    assert o.mode == hf.HF_MODE_PERSISTENT and o.priority == hf.HF_PRIO_FIFO
    assert o.claim == 8 and o.local_keep == -1 and o.stall_task == -1
    for s in range(9):
        assert hf.hf_status_string(s).startswith(hf.STATUS_NAMES[s])


def _status(fn, *args):
    try:
        fn(*args)
    except hf.HfError as e:
        return e.status
    return hf.HF_OK


def test_builder_levels_match_networkx():
    g = S.layered(5, 3000, 25, 1, 4)
    h = hf.hf_graph_create(g.n, g.m)
    assert hf.hf_add_tasks_bulk(h, g.n) == 0
    hf.hf_precede_bulk(h, g.src, g.dst, g.delay)
    hf.hf_finalize(h)
    info = hf.hf_graph_info(h)
    assert info["tasks"] == g.n and info["edges"] == g.m and info["levels"] == 25 and info["finalized"]
    assert info["sources"] == 3000 // 25 and info["kind_count"][hf.HF_KERNEL] == g.n
    lev = hf.hf_get_levels(h, g.n)
    G = nx.DiGraph()
    G.add_nodes_from(range(g.n))
    G.add_edges_from(zip(g.src.tolist(), g.dst.tolist()))
    ref = np.zeros(g.n, np.int32)
    for k, gen in enumerate(nx.topological_generations(G)):
        ref[list(gen)] = k
    np.testing.assert_array_equal(lev, ref)
    hf.hf_graph_destroy(h)


def test_cycle_and_self_loop_are_reported():
    h = hf.hf_graph_create()
    hf.hf_add_tasks_bulk(h, 4)
    hf.hf_precede(h, 0, 1)
    hf.hf_precede(h, 1, 2)
    hf.hf_precede(h, 2, 1)
    assert _status(hf.hf_finalize, h) == hf.HF_ECYCLE
    assert "cycle" in hf.hf_last_error()
    hf.hf_graph_destroy(h)
    h = hf.hf_graph_create()
    hf.hf_add_tasks_bulk(h, 2)
    hf.hf_precede(h, 1, 1)
    assert _status(hf.hf_finalize, h) == hf.HF_ECYCLE
    hf.hf_graph_destroy(h)


def test_invalid_arguments():
    h = hf.hf_graph_create()
    hf.hf_add_tasks_bulk(h, 3)
    assert _status(hf.hf_precede, h, 0, 3) == hf.HF_EINVAL
    assert _status(hf.hf_precede, h, -1, 0) == hf.HF_EINVAL
    assert _status(hf.hf_precede_w, h, 0, 1, float("nan")) == hf.HF_EINVAL
    assert _status(hf.hf_precede_w, h, 0, 1, float("inf")) == hf.HF_EINVAL
    # bulk is all-or-nothing
    assert _status(hf.hf_precede_bulk, h, [0, 1], [1, 7], [1.0, 1.0]) == hf.HF_EINVAL
    assert hf.hf_graph_info(h)["edges"] == 0
    assert _status(hf.hf_add_task, h, 9, None) == hf.HF_EINVAL
    mp = hf.hf_maxplus_payload(op=hf.HF_K_MAXPLUS, arr0=float("nan"))
    assert _status(hf.hf_add_task, h, hf.HF_KERNEL, mp) == hf.HF_EINVAL
    # a saxpy whose x "pull" is not a pull task, or has no buffer at all
    sp = hf.hf_saxpy_payload(op=hf.HF_K_SAXPY_F32, n=16, x_pull=0, y_pull=-1, y_dev=256)
    assert _status(hf.hf_add_task, h, hf.HF_KERNEL, sp) == hf.HF_EINVAL
    sp = hf.hf_saxpy_payload(op=hf.HF_K_SAXPY_F32, n=16, x_pull=-1, y_pull=-1, y_dev=256)
    assert _status(hf.hf_add_task, h, hf.HF_KERNEL, sp) == hf.HF_EINVAL
    # pull buffer smaller than the saxpy operand
    buf = np.zeros(8, np.float32)
    pl = hf.hf_add_task(h, hf.HF_PULL, hf.hf_pull_payload(host_ptr=buf.ctypes.data, bytes=32))
    sp = hf.hf_saxpy_payload(op=hf.HF_K_SAXPY_F32, n=16, x_pull=pl, y_pull=-1, y_dev=256)
    assert _status(hf.hf_add_task, h, hf.HF_KERNEL, sp) == hf.HF_EINVAL
    sp.n = 8
    assert hf.hf_add_task(h, hf.HF_KERNEL, sp) == pl + 1
    # push from a task that is not a pull
    ps = hf.hf_push_payload(src_pull=0, host_ptr=buf.ctypes.data, bytes=4)
    assert _status(hf.hf_add_task, h, hf.HF_PUSH, ps) == hf.HF_EINVAL
    ps = hf.hf_push_payload(src_pull=pl, host_ptr=buf.ctypes.data, bytes=64)
    assert _status(hf.hf_add_task, h, hf.HF_PUSH, ps) == hf.HF_EINVAL
    info = hf.hf_graph_info(h)
    assert info["kind_count"][hf.HF_PULL] == 1 and info["payload_tasks"] == 2
    hf.hf_graph_destroy(h)


def test_batch_membership_blocks_mutation():
    h = hf.hf_graph_create()
    hf.hf_add_tasks_bulk(h, 2)
    hf.hf_precede(h, 0, 1)
    b = hf.hf_batch_create()
    assert hf.hf_batch_add(b, h) == 0
    assert _status(hf.hf_precede, h, 0, 1) == hf.HF_ESTATE
    assert _status(hf.hf_graph_destroy, h) == hf.HF_ESTATE
    hf.hf_batch_destroy(b)
    hf.hf_precede(h, 0, 1)
    hf.hf_graph_destroy(h)


def test_paper_dependency_graph_levels():
    from golden_io import load

    gold = load("paper_dependency_graph.txt")
    names = [t[0] for t in gold["tasks"]]
    ix = {nm: i for i, nm in enumerate(names)}
    h = hf.hf_graph_create()
    hf.hf_add_tasks_bulk(h, len(names))
    for a, b in gold["edges"]:
        hf.hf_precede(h, ix[a], ix[b])
    hf.hf_finalize(h)
    lev = hf.hf_get_levels(h, len(names))
    for a, b in gold["edges"]:
        assert lev[ix[a]] < lev[ix[b]]
    assert lev[ix["kernel2"]] == 3 and lev[ix["push2"]] == 4 and hf.hf_graph_info(h)["levels"] == 5
    hf.hf_graph_destroy(h)
