"""Row-group checkpoint / resume (Fig. 18 Stage 2 resume manifest), on the CPU
with a stand-in propagator: the field of rows [j0, j1) is a deterministic sum
of per-row fields, so a resumed run must reproduce the uninterrupted one."""
import json
import os

import numpy as np
import pytest

from paper_2609_01978_gb300 import resume as R

M = 8


def row_field(j):
    rng = np.random.default_rng(1000 + j)
    return rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))


class Source:
    def __init__(self):
        self.calls = []

    def __call__(self, j0, j1):
        self.calls.append((j0, j1))
        return sum(row_field(j) for j in range(j0, j1))


PARAMS = {"D": 0.25, "f": 1.25, "lambda": 632.8e-9, "N": 101, "M": M}


def test_full_run_is_the_sum_of_rows(tmp_path):
    src = Source()
    run = R.GroupRun(str(tmp_path), PARAMS, M, 10, 91, 16)
    U = run.run(src)
    ref = sum(row_field(j) for j in range(10, 91))
    assert np.max(np.abs(U - ref)) < 1e-12
    assert src.calls == R.groups(10, 91, 16) and src.calls[-1] == (90, 91)
    m = json.load(open(os.path.join(tmp_path, R.MANIFEST)))
    assert sorted(int(k) for k in m["done"]) == list(range(6))


def test_interrupted_run_resumes_where_it_stopped(tmp_path):
    src = Source()

    def stop_after_two(k):
        if k == 1:
            raise KeyboardInterrupt

    with pytest.raises(KeyboardInterrupt):
        R.GroupRun(str(tmp_path), PARAMS, M, 0, 101, 20).run(src, on_group=stop_after_two)
    assert len(src.calls) == 2
    src2 = Source()
    U = R.GroupRun(str(tmp_path), PARAMS, M, 0, 101, 20).run(src2)
    assert src2.calls == R.groups(0, 101, 20)[2:]
    ref = sum(row_field(j) for j in range(0, 101))
    assert np.max(np.abs(U - ref)) < 1e-12


def test_corrupted_group_is_recomputed(tmp_path):
    run = R.GroupRun(str(tmp_path), PARAMS, M, 0, 40, 10)
    run.run(Source())
    path = os.path.join(tmp_path, "group_000002.npy")
    a = np.load(path)
    a[0, 0] += 1.0
    np.save(path, a)
    run2 = R.GroupRun(str(tmp_path), PARAMS, M, 0, 40, 10)
    assert run2.pending() == [2]
    src = Source()
    U = run2.run(src)
    assert src.calls == [(20, 30)]
    assert np.max(np.abs(U - sum(row_field(j) for j in range(40)))) < 1e-12


def test_foreign_manifest_is_refused(tmp_path):
    R.GroupRun(str(tmp_path), PARAMS, M, 0, 40, 10).run(Source())
    with pytest.raises(ValueError):
        R.GroupRun(str(tmp_path), dict(PARAMS, D=0.3), M, 0, 40, 10)
    with pytest.raises(ValueError):
        R.GroupRun(str(tmp_path), PARAMS, M, 0, 40, 20)


def test_preflight_refuses_a_full_disk(tmp_path, monkeypatch):
    run = R.GroupRun(str(tmp_path), PARAMS, M, 0, 40, 10)

    class Usage:
        total, used, free = 1 << 20, 1 << 20, 100

    monkeypatch.setattr(R.shutil, "disk_usage", lambda p: Usage)
    with pytest.raises(OSError):
        run.run(Source())
