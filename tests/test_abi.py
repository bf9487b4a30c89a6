"""The C-ABI library builds for sm_103a, loads, and exports every entry
point include/coremaint.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "coremaint.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cm_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def so():
    from paper_1612_09368_gb300 import build
    return build.build()


def test_library_exports_every_declared_entry_point(so):
    lib = ctypes.CDLL(so)
    names = declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_struct_layouts_match_header():
    import paper_1612_09368_gb300 as cm
    # cm_options: 6 int32, int64, 3 pointers, 12 int32
    assert ctypes.sizeof(cm.cm_options) == 6 * 4 + 8 + 3 * 8 + 12 * 4
    assert ctypes.sizeof(cm.cm_step_config) == 8 * 4
    # cm_stats: 14 int64, 2 double, peel_levels, barriers, grid_iterations, phase_ns[7], reserved[4]
    assert ctypes.sizeof(cm.cm_stats) == 14 * 8 + 2 * 8 + (3 + 7 + 4) * 8
    # cm_check_report: 8 int64 (vertices checked, five mismatch counts, first bad vertex, reserved)
    assert ctypes.sizeof(cm.cm_check_report) == 8 * 8


def test_default_options_without_gpu(so):
    import paper_1612_09368_gb300 as cm
    o = cm.cm_default_options()
    assert (o.slack_pct, o.min_cap, o.block_threads, o.spin_limit_ns) == (25, 4, 512, 4_000_000_000)
    assert (o.block_mode_edges, o.block_mode_enter, o.block_mode_leave) == (16384, 1024, 8192)
    assert (o.hub_slots, o.block_slots, o.block_slots_delete, o.task_claim) == (1024, 4096, 1024, 1)
    assert (o.select_order, o.select_rounds) == (cm.CM_SELECT_HASH, 0)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import paper_1612_09368_gb300 as cm
    monkeypatch.setattr(cm, "_lib", None)
    monkeypatch.setattr(cm, "library_path", str(tmp_path / "absent.so"))
    with pytest.raises(ImportError):
        cm.lib()
