"""hf_dump writes the graph as Graphviz DOT (host only): every task once with its kind, every
dependency once with its delay, round-tripping binary32."""
import re

import numpy as np

from paper_2203_08395_b300 import build as B
from paper_2203_08395_b300 import hf


def test_dump_lists_tasks_kinds_and_delays(tmp_path):
    B.build()
    g = hf.hf_graph_create()
    a = hf.hf_add_task(g, hf.HF_KERNEL, hf.hf_maxplus_payload(op=hf.HF_K_MAXPLUS, arr0=-2.5))
    b = hf.hf_add_task(g, hf.HF_KERNEL, None)
    c = hf.hf_add_task(g, hf.HF_KERNEL, hf.hf_saxpy_payload(op=hf.HF_K_SAXPY_F32, a_f=2.0, n=77, x_pull=-1,
                                                           y_pull=-1, x_dev=16, y_dev=32))
    first = hf.hf_add_tasks_bulk(g, 3)
    delays = np.array([0.1, 1e-7, 3.0, 0.75, 2.5], np.float32)
    edges = [(a, b), (a, c), (b, first), (c, first + 1), (first + 1, first + 2)]
    for (u, v), d in zip(edges, delays):
        hf.hf_precede_w(g, u, v, float(d))
    path = tmp_path / "g.dot"
    hf.hf_dump(g, str(path))
    text = path.read_text()
    assert text.startswith("digraph") and text.rstrip().endswith("}")
    nodes = dict((int(i), lab) for i, lab in re.findall(r'^\s*t(\d+) \[label="([^"]*)"\];$', text, re.M))
    got = [(int(u), int(v), np.float32(float(d))) for u, v, d in
           re.findall(r'^\s*t(\d+) -> t(\d+) \[label="([^"]*)"\];$', text, re.M)]
    assert sorted(nodes) == list(range(6))
    assert nodes[a] == "0 maxplus arr0=-2.5" and nodes[c] == "2 saxpy n=77" and nodes[b].startswith("1 maxplus")
    assert got == [(u, v, d) for (u, v), d in zip(edges, delays)]
    hf.hf_graph_destroy(g)
