"""Host-side checks of the C ABI: the library builds for sm_103a, loads, exports every
entry point include/pcv.h declares, and rejects calls it can reject without a GPU."""
import ctypes
import re
from pathlib import Path

import pytest

from paper_1801_02362_gb300 import build_lib, pcv

ROOT = Path(__file__).resolve().parents[1]
HEADER = ROOT / "include" / "pcv.h"


def declared_symbols():
    text = HEADER.read_text()
    return sorted(set(re.findall(r"^PCV_API\s+[\w\s\*]+?\b(pcv_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return pcv.load()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("pcv_create", "pcv_destroy", "pcv_set_landmarks", "pcv_set_lambda", "pcv_set_close_threshold",
                     "pcv_evaluate", "pcv_evaluate_host", "pcv_reset_close_state", "pcv_save_state",
                     "pcv_load_state", "pcv_get_stats", "pcv_sync", "pcv_last_error", "pcv_combine_grad"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(declared_symbols()) <= set(pcv.SIGNATURES)


def test_build_targets_sm_103a_only(monkeypatch, tmp_path):
    """Every nvcc command of the build (each translation unit and the link) carries the one
    -gencode for sm_103a and no other architecture.  The commands are recorded by a stand-in
    for subprocess.run that creates the outputs it is asked for."""
    cmds = []

    class Done:
        returncode, stdout, stderr = 0, "", ""

    def fake_run(cmd, **kw):
        cmds.append(list(cmd))
        Path(cmd[cmd.index("-o") + 1]).write_bytes(b"")
        return Done()

    monkeypatch.setattr(build_lib.subprocess, "run", fake_run)
    monkeypatch.setattr(build_lib, "BUILD", tmp_path)
    monkeypatch.setattr(build_lib, "LIB", tmp_path / "libpcv.so")
    build_lib.build(force=True)
    assert len(cmds) == len(build_lib.SOURCES) + 1
    for cmd in cmds:
        gencodes = [cmd[k + 1] for k, a in enumerate(cmd) if a == "-gencode"]
        assert gencodes == ["arch=compute_103a,code=sm_103a"], cmd
        assert not any(a.startswith(("-arch", "--gpu-architecture")) for a in cmd), cmd


def test_null_context_is_rejected_without_gpu(lib):
    assert lib.pcv_set_lambda(None, 1.0) == pcv.PCV_EINVAL
    assert lib.pcv_evaluate(None, 1, None, None, None, None, None, None, None) == pcv.PCV_EINVAL
    assert lib.pcv_destroy(None) == pcv.PCV_OK
    assert isinstance(lib.pcv_last_error(None), bytes)
    st = pcv.pcv_stats()
    assert ctypes.sizeof(st) == 9 * 8


def test_create_reports_bad_precision(lib):
    h = ctypes.c_void_p()
    assert lib.pcv_create(ctypes.byref(h), 0, None, 7) == pcv.PCV_EINVAL
    assert h.value is None


def test_new_entry_points_reject_null_without_gpu(lib):
    assert lib.pcv_set_neighbor_list(None, 5, 5) == pcv.PCV_EINVAL
    assert lib.pcv_metad_apply(None, 1, 1, 1, None, None, None, None, None, None) == pcv.PCV_EINVAL
    assert lib.pcv_metad_destroy(None) == pcv.PCV_OK
    assert isinstance(lib.pcv_metad_last_error(None), bytes)
    h = ctypes.c_void_p()
    assert lib.pcv_metad_create(ctypes.byref(h), 0, None, 1.0, 0.0, 1.0, 1, 10) == pcv.PCV_EINVAL
    assert h.value is None


def test_host_chunk_plan(lib):
    """The chunk plan of pcv_evaluate_host (host logic, no device): the chunks cover the
    batch in order, each holds at least 2048 frames, the count follows the option (or about
    one chunk per 16k frames, at most 8), and the first and last chunk hold end_share percent
    of a middle one unless the 2048-frame floor lifts them."""
    for F in (1, 2047, 4096, 9000, 16384, 16385, 100000, 1000003):
        for n, e in ((0, 25), (1, 25), (2, 25), (3, 100), (4, 1), (7, 25), (8, 100), (64, 50)):
            plan = pcv.pcv_host_chunk_plan(F, n, e)
            want_n = n if n > 0 else min(8, max(1, -(-F // 16384)))
            want_n = min(want_n, max(1, F // 2048))
            assert len(plan) == want_n, (F, n, e, plan)
            assert sum(plan) == F and all(x > 0 for x in plan)
            if len(plan) > 1:
                assert min(plan) >= 2048, (F, n, e, plan)
            if len(plan) >= 3:
                mid = plan[1]
                assert max(plan[1:-1]) - min(plan[1:-1]) <= 1
                assert plan[0] == plan[-1]
                assert plan[0] == max(2048, int(F / ((len(plan) - 2) + 2 * e / 100) * e / 100)), (F, n, e, plan)
                assert plan[0] <= mid + 1
    assert pcv.pcv_host_chunk_plan(0) == []
    for bad in ((-1, 0, 25), (10, -1, 25), (10, 65, 25), (10, 0, 0), (10, 0, 101)):
        with pytest.raises(pcv.PcvError) as err:
            pcv.pcv_host_chunk_plan(*bad)
        assert err.value.status == pcv.PCV_EINVAL
