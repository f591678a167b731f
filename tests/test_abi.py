"""The CUDA library builds, loads and exports exactly the C ABI that
include/flowroi.h declares; host-only entry points work without a GPU
(no kernel is launched here)."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def F():
    from paper_2511_14419_gb300 import build, flowroi
    build()
    return flowroi


def _declared():
    src = open(os.path.join(ROOT, "include", "flowroi.h")).read()
    return sorted(set(re.findall(r"FLOWROI_API\s+[\w\s\*]*?\b(flowroi_\w+)\s*\(", src)))


def test_header_declares_the_abi():
    names = _declared()
    assert "flowroi_create" in names and "flowroi_submit_frame" in names and "flowroi_get_mask" in names
    assert len(names) >= 14


def test_library_exports_every_declared_symbol(F):
    out = subprocess.run(["nm", "-D", "--defined-only", F.LIB], capture_output=True, text=True, check=True).stdout
    exported = sorted({ln.split()[-1] for ln in out.splitlines() if " T " in ln})
    assert exported == _declared()
    L = F.lib()
    for name in _declared():
        assert hasattr(L, name)
    assert sorted(F.EXPORTS) == _declared()


def test_struct_sizes_match_binding(F):
    import ctypes
    cfg = F.flowroi_default_config()
    assert cfg.struct_size == ctypes.sizeof(F.flowroi_config)
    assert (cfg.roi_q, cfg.scale_shift, cfg.win_r, cfg.iters) == (np.float32(0.2), 5, 7, 3)
    assert F.flowroi_abi_version() == 6
    assert ctypes.sizeof(F.flowroi_cs_job) == 72


def test_quant_steps_match_oracle_table(F, orc):
    for levels, bd in [(5, 12), (3, 8), (1, 12), (6, 16)]:
        d, e, m, g = F.flowroi_quant_steps(levels, bd, 1.0)
        G, dd, ee, mm = orc.delta_table(levels, bd, 1.0)
        assert np.array_equal(d, dd) and np.array_equal(e, ee) and np.array_equal(m, mm)
        assert np.max(np.abs(g / G - 1)) < 1e-12


def test_config_validation_is_host_side(F):
    bad = [dict(roi_q=0.0), dict(roi_q=1.0), dict(wavelet=44), dict(win_r=1), dict(win_r=11), dict(poly_n_half=4),
           dict(lam=0.0), dict(r_open=5), dict(precision=8), dict(max_batch_frames=0), dict(result_ring=1),
           dict(dwt_levels=9), dict(scale_shift=16), dict(flags=0x80), dict(codestream_reset=2)]
    for kw in bad:
        cfg = F.flowroi_default_config(**kw)
        with pytest.raises(F.FlowRoIError) as ei:
            F.flowroi_create(cfg)
        assert ei.value.code == F.EINVAL, kw
    cfg = F.flowroi_default_config()
    cfg.struct_size = 4
    with pytest.raises(F.FlowRoIError):
        F.flowroi_create(cfg)


def test_null_context_is_rejected(F):
    import ctypes
    L = F.lib()
    assert L.flowroi_step(None) == F.EINVAL
    assert L.flowroi_flush(None, 0) == F.EINVAL
    assert L.flowroi_end_stream(None, 1) == F.EINVAL
    buf = np.zeros(4, np.uint8)
    assert L.flowroi_get_mask(None, 0, 0, buf.ctypes.data, 0, 0) == F.EINVAL
    L.flowroi_destroy(None)
    assert isinstance(L.flowroi_last_error(None), bytes)
    del ctypes


def test_log_env_reports_refusals_on_stderr():
    """FLOWROI_LOG=1 logs every refusal (here a config error, which needs no
    GPU) to stderr; without it the library is silent."""
    import subprocess
    import sys
    code = ("from paper_2511_14419_gb300 import flowroi as F\n"
            "try:\n    F.Context(roi_q=2.0)\nexcept F.FlowRoIError:\n    pass\n")
    env = dict(os.environ, FLOWROI_LOG="1")
    on = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, cwd=ROOT, timeout=120)
    assert "[flowroi] status -1: config.roi_q" in on.stderr, on.stderr
    env.pop("FLOWROI_LOG")
    off = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, cwd=ROOT, timeout=120)
    assert "[flowroi]" not in off.stderr


def test_codestream_bound_counts_the_code_blocks(F, orc):
    """The bound covers both formats: the JPEG2000 codestream's markers
    (256 bytes) + per code-block its packet-header bits (at most 192 bytes)
    and the coder's per-block byte limit, which exceeds the container's
    header + per code-block entry, pass lengths and bytes; the library's
    code-block count agrees with the oracle's partition; malformed
    geometries give 0."""
    for w, h, levels in [(2048, 2048, 5), (256, 256, 3), (264, 200, 3), (16, 16, 2), (2048, 1536, 5)]:
        n = len(orc.codeblocks(w, h, levels))
        b = F.flowroi_codestream_bound(w, h, levels)
        assert b == 256 + n * (192 + 32768)
        assert b >= 32 + n * (16 + 2 * 70 + 32768)
    for w, h, levels in [(100, 64, 3), (64, 64, 0), (64, 64, 9), (0, 64, 1), (65536, 64, 1)]:
        assert F.flowroi_codestream_bound(w, h, levels) == 0


def test_get_results_rejects_bad_arguments_on_the_host(F):
    L = F.lib()
    assert L.flowroi_get_results(None, 1, None, None, None, None, 0, 0, None) == F.EINVAL
    assert "ctx is NULL" in F.flowroi_last_error(None)


def test_encode_codestreams_rejects_bad_jobs_on_the_host(F):
    L = F.lib()
    jobs = (F.flowroi_cs_job * 1)()
    assert L.flowroi_encode_codestreams(None, 1, jobs, 0) == F.EINVAL
    import ctypes
    n = ctypes.c_uint64(0)
    assert L.flowroi_get_codestream(None, 0, 0, jobs, 0, ctypes.byref(n), 0, 0) == F.EINVAL
