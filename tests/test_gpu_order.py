"""Kernel order in a fresh process: the benchmark's sequence (instrumented team runs with
payloads recording task costs, an instrumented persistent run, cost-model training and
evaluation, then the machine-constant calibration, the prediction and a team run). Shared
memory is not cleared between kernels, so the first team launches of a process run on whatever
the earlier kernels left there; this runs them after the cost-model kernels, as the benchmark
does, in a process of its own (calibration happens once per process)."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CODE = textwrap.dedent("""
    import numpy as np, torch
    import oracle
    from paper_2203_08395_b300 import hf, learn, synth as S
    from paper_2203_08395_b300.workload import BatchOnDevice
    hf.load(); hf.install_torch_allocator()
    stream = torch.cuda.current_stream()
    wl = S.batch(7, graphs=24, nmin=1000, nmax=40000, frac_saxpy=0.1)
    bd = BatchOnDevice(wl)
    train = [BatchOnDevice(S.batch(s, graphs=16, nmin=1000, nmax=40000, frac_saxpy=0.1)) for s in (101, 102)]
    recs = [learn.record(tb, stream) for tb in train] + [learn.record(train[0], stream, executor="persistent")]
    for tb in train:
        tb.close()
    cm = hf.hf_costmodel_create(0)
    learn.train(cm, recs, rows=65536, epochs=4)
    learn.evaluate(bd, cm, learn.record(bd, stream), stream)
    hf.hf_batch_set_costmodel(bd.b, cm)
    hf.hf_calibration(stream)
    hf.hf_batch_predict(bd.b, hf.HF_PRIO_LEARNED, stream)
    for o in (dict(mode=hf.HF_MODE_TEAM, priority=hf.HF_PRIO_LEARNED), dict(mode=hf.HF_MODE_TEAM, team_size=1)):
        bd.run(stream, **o)
        bd.sync()
        for i, g in enumerate(wl.graphs):
            a = bd.arrivals(i).view(np.uint32)
            assert np.array_equal(a, oracle.run_spec(g)["arr"].view(np.uint32)), (o, i)
    print("order ok")
""")


def test_calibration_and_team_runs_after_cost_model_training():
    r = subprocess.run([sys.executable, "-c", CODE], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "order ok" in r.stdout, (r.stdout[-2000:] + r.stderr[-4000:])
