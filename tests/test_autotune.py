"""Host logic of the launch-shape autotuner: problem signatures, range checks
of table entries, table lookup and how an entry is applied to an instance
(a recording stand-in for the instance; no GPU)."""
import json
import os
import re

import pytest

from paper_1709_05660_gb300 import autotune
from paper_1709_05660_gb300.workloads import CONFIGS, SolverOpts, problem_3d

ENTRY = {"levels": {"1": dict(apply_slices=8, apply_groups=32, spmv_sub=8),
                    "2": dict(apply_slices=1, apply_groups=4, spmv_sub=4)},
         "gj_panel": 32}


def test_signature_fixes_block_shapes_not_materials():
    prob, opts = CONFIGS["channel2d_l5"]
    assert autotune.signature(prob, opts) == "2d-L5-c16x4-t4x4-fp64"
    from dataclasses import replace
    soft = replace(prob, mu_s=1e4, U=0.1)
    assert autotune.signature(soft, replace(opts, precision=1)) == "2d-L5-c16x4-t4x4-mixed"
    assert autotune.signature(problem_3d(levels=2), SolverOpts(tile=(2, 2, 2))) == "3d-L2-c16x4x4-t2x2x2-fp64"


def test_check_entry_ranges():
    autotune.check_entry(ENTRY, 3)
    with pytest.raises(ValueError):
        autotune.check_entry(ENTRY, 2)                      # level 2 does not exist
    for bad in (dict(apply_slices=0, apply_groups=4, spmv_sub=4), dict(apply_slices=2, apply_groups=300, spmv_sub=4),
                dict(apply_slices=2, apply_groups=4, spmv_sub=3)):
        with pytest.raises(ValueError):
            autotune.check_entry({"levels": {"1": bad}}, 3)
    with pytest.raises(ValueError):
        autotune.check_entry({"levels": {}, "gj_panel": 20}, 3)


def test_lookup_by_gpu_and_signature():
    prob, opts = CONFIGS["channel2d_l3"]
    table = {"GPU A": {autotune.signature(prob, opts): ENTRY}}
    assert autotune.lookup(prob, opts, gpu="GPU A", table=table) is ENTRY
    assert autotune.lookup(prob, opts, gpu="GPU B", table=table) is None
    from dataclasses import replace
    assert autotune.lookup(prob, replace(opts, tile=(4, 4)), gpu="GPU A", table=table) is None


class _Recorder:
    def __init__(self, prob, opts):
        self.prob, self.opts, self.calls = prob, opts, []

    def set_launch_params(self, level, **kw):
        self.calls.append((level, kw))


def test_apply_table_sets_every_level_and_the_panel_on_the_finest():
    prob, opts = CONFIGS["channel2d_l3"]          # 3 levels: Schwarz levels 1 and 2
    rec = _Recorder(prob, opts)
    assert autotune.apply_table(rec, ENTRY) is ENTRY
    assert rec.calls == [(1, dict(apply_slices=8, apply_groups=32, spmv_sub=8, gj_panel=0)),
                         (2, dict(apply_slices=1, apply_groups=4, spmv_sub=4, gj_panel=32))]
    rec = _Recorder(prob, opts)
    assert autotune.apply_table(rec, {}) is None and rec.calls == []


def test_committed_table_is_valid():
    if not os.path.exists(autotune.TABLE):
        pytest.skip("no tuning table committed")
    table = json.load(open(autotune.TABLE))
    assert table
    for gpu, entries in table.items():
        for sig, entry in entries.items():
            m = re.fullmatch(r"([23])d-L(\d+)-c[\dx]+-t[\dx]+-(mixed|fp64)", sig)
            assert m, sig
            autotune.check_entry(entry, int(m.group(2)))
            assert set(entry["levels"]) == {str(l) for l in range(1, int(m.group(2)))}, sig
