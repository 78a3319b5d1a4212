"""The oracle's pins must catch plausible mistakes: each mutant below is the oracle's source
with one planted error (compiled on the CPU into a temporary library); running the pins
against it must fail. Mistakes planted only in the oracle, never in GPU code."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import test_oracle_kahn as pins

MUTANTS = {
    "plain_less_instead_of_total_order": ("if (below(arr[v], cand))", "if (arr[v] < cand)"),
    "subtract_delay": ("arr[u] + delay[e]", "arr[u] - delay[e]"),
    # released once, but while one predecessor is still pending (single-predecessor tasks never run)
    "release_one_early": ("if (--pending[v] == 0)", "if (--pending[v] == 1)"),
    "ignore_source_arrival": ("arr[v] = arr0 ? arr0[v] : 0.0f;", "arr[v] = 0.0f;"),
    "saxpy_operands_swapped": ("y[i] = fmaf(a, x[i], y[i]);", "y[i] = fmaf(a, y[i], x[i]);"),
    "max_keeps_first": ("if (below(arr[v], cand)) arr[v] = cand;",
                        "if (arr[v] == -INFINITY) arr[v] = cand;"),
}


def _build_mutant(tmpdir, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "kahn.c")).read()
    assert src.count(old) >= 1, name
    path_c = os.path.join(tmpdir, name + ".c")
    path_so = os.path.join(tmpdir, name + ".so")
    open(path_c, "w").write(src.replace(old, new))
    subprocess.check_call(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                           "-o", path_so, path_c, "-lm"])
    return path_so


def _all_pins():
    fns = [pins.test_bruteforce_paths_bit_exact_1000_tiny_dags, pins.test_negative_zero_is_below_positive_zero,
           pins.test_every_task_once_after_all_predecessors, pins.test_saxpy_f32_closed_forms,
           pins.test_chain_is_fp32_prefix_sum]
    failed = []
    for f in fns:
        try:
            f()
        except AssertionError:
            failed.append(f.__name__)
    return failed


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, monkeypatch):
    with tempfile.TemporaryDirectory() as d:
        so = _build_mutant(d, name, *MUTANTS[name])
        saved = oracle.lib()
        L = ctypes.CDLL(so)
        L.oracle_kahn.argtypes = saved.oracle_kahn.argtypes
        L.oracle_kahn.restype = saved.oracle_kahn.restype
        L.oracle_saxpy_f32.argtypes = saved.oracle_saxpy_f32.argtypes
        L.oracle_saxpy_f32.restype = None
        monkeypatch.setattr(oracle, "_lib", L)
        failed = _all_pins()
    assert failed, "mutant %s passed every pin" % name
