"""Host-side checks that need no GPU: the library loads and exports every
entry point declared in include/emugemm.h, its method constants agree with
the oracle's independent derivations, argument validation, the
multi-rank aggregation of bench.py over a 2-rank gloo process group, and
the JSON line of the benchmark's reference arm (the oracle on the host)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "emugemm.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_25453_gb300 as emu
    return emu


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(emu_[A-Za-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 35
    missing = [n for n in names if not hasattr(lib.lib, n)]
    assert not missing, missing


def test_constants_match_oracle(lib, orc):
    for p in range(1, 13):
        assert lib.emu_chunk_len_I(p) == orc.chunk_len_I(p)
    assert lib.moduli(20) == orc.moduli(20)
    for nm in (1, 5, 12, 16, 20):
        for k in (1, 100, 4096, 8192, 131071):
            for c in (0, 1):
                assert lib.emu_scale_bits_II(nm, k, c) == orc.scale_bits_II(nm, k, bool(c))


def test_split_layout_sizes(lib):
    assert lib.emu_split_rows(1) == 128 and lib.emu_split_rows(129) == 256
    assert lib.emu_split_cols_I(33, 3) == 64 * 3
    assert lib.emu_split_cols_II(129) == 256


def test_argument_validation_without_gpu(lib):
    sz = ctypes.c_size_t()
    assert lib.emu_workspace_size(1, 100, 100, 100, 8, 0, ctypes.byref(sz)) == 0 and sz.value > 2 * 100 * 800
    assert lib.emu_workspace_size(1, 10, 10, 10, 13, 0, ctypes.byref(sz)) == 2
    assert lib.emu_workspace_size(2, 10, 10, 10, 21, 0, ctypes.byref(sz)) == 2
    assert lib.emu_workspace_size(3, 10, 10, 10, 5, 0, ctypes.byref(sz)) == 0  # E4M3 slices
    assert lib.emu_workspace_size(4, 10, 10, 10, 5, 0, ctypes.byref(sz)) == 0  # Scheme II, norm scaling
    assert lib.emu_workspace_size(5, 10, 10, 10, 5, 0, ctypes.byref(sz)) == 1
    assert lib.emu_dgemm(None, 0, 4, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4, 1, 3, None) == 1
    assert lib.emu_status_string(6) == b"EMU_ERR_TIMEOUT"
    # column-major leading dimensions must cover the rows
    assert lib.emu_dgemm_noalloc(1, 8, 8, 8, 1.0, 1, 4, 1, 8, 0.0, 1, 8, 4, None, None) == 1
    # complex Scheme I workspace covers the 2K-deep embedding; CGEMM needs a handle
    assert lib.emu_workspace_size(1, 100, 100, 100, 8, 1, ctypes.byref(sz)) == 0 and sz.value > 16 * 300 * 100
    lib.emu_cgemm.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                              ctypes.c_void_p]
    one = (ctypes.c_float * 2)(1.0, 0.0)
    assert lib.emu_cgemm(None, 0, 4, 4, 4, one, None, 4, None, 4, one, None, 4, 1, 4, None) == 1
    # the separate epilogue rejects a null handle and short leading dimensions
    lib.emu_shift_reduce_I.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    assert lib.emu_shift_reduce_I(None, 4, 4, 8, 0, 1, 1, 1, 1.0, 0.0, 1, 4, None) == 1


def test_create_without_gpu_reports_cuda_error(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.emu_create(ctypes.byref(h), 0) == 4  # EMU_ERR_CUDA


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank  # the slower rank decides
    mx = bench.max_over_ranks(ms, dist, "cpu")
    val = bench.aggregate_tflops(world, 2.0 * 8192 ** 3, 5, mx)
    out[rank] = (mx, val)
    dist.destroy_process_group()


def test_multirank_aggregation_gloo():
    import socket
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mgr = mp.get_context("spawn").Manager()  # no fork of this multi-threaded process
    out = mgr.dict()
    mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
    assert out[0][0] == out[1][0] == 150.0
    expect = 2 * 2.0 * 8192 ** 3 * 5 / 0.150 / 1e12
    assert abs(out[0][1] - expect) < 1e-9 * expect


def test_suite_markdown_tables(tmp_path):
    # the summary of a --suite file: engine tables, speedups against the
    # INT8 engine and against cuBLAS SGEMM, bits = -log2 of the sampled error
    import json

    import bench
    rows = [
        {"path": "cublas_sgemm", "n": 8192, "tflops": 70.0, "ms": 15.7, "err": 2.0 ** -22},
        {"path": "emu_dgemm_II", "n": 8192, "phi": 0.5, "nm": 16, "tflops": 62.0, "engine": "bf16 tcgen05",
         "tensor_tops": 992.0, "ms": 17.7, "err": 2.0 ** -56},
        {"path": "emu_dgemm_II_int8", "n": 8192, "phi": 0.5, "nm": 16, "tflops": 8.7, "engine": "int8 mma.sync",
         "tensor_tops": 139.0, "ms": 126.4, "err": 2.0 ** -56},
        {"path": "emu_sgemm_II", "n": 8192, "phi": 0.5, "nm": 8, "tflops": 116.0, "tensor_tops": 928.0, "ms": 9.5,
         "err": 2.0 ** -24},
    ]
    path = tmp_path / "s.jsonl"
    path.write_text("".join(json.dumps(r) + "\n" for r in rows))
    md = bench.suite_markdown(str(path))
    assert "| 8192 | 0.5 | 16 | 62.000 | 992.0 | 56.0 |" in md
    assert "| 8192 | 0.5 | 16 | 8.700 | 139.0 | 56.0 | 7.14x |" in md
    assert "| 8 | 116.00 | 24.0 | 1.66x |" in md
    # a later file (a --suite-part scheme2 run) replaces the matching rows only
    later = tmp_path / "s2.jsonl"
    later.write_text(json.dumps(dict(rows[1], tflops=64.0, ms=17.2, tensor_tops=1023.0)) + "\n")
    md2 = bench.suite_markdown([str(path), str(later)])
    assert "| 8192 | 0.5 | 16 | 64.000 | 1023.0 | 56.0 |" in md2 and "| 8192 | 0.5 | 16 | 62.000 |" not in md2
    assert "| 8192 | 0.5 | 16 | 8.700 | 139.0 | 56.0 | 7.35x |" in md2  # against the replaced row
    assert "| 8 | 116.00 | 24.0 | 1.66x |" in md2 and "replace the rows of earlier files" in md2


def test_selector_markdown(tmp_path):
    # the end-to-end selector summary: per (scheme, tol) totals, speed-up and pass rates
    import json

    import bench
    rows = [
        {"path": "selector_e2e", "scheme": "I", "n": 2048, "phi": 1.0, "tol": 1e-8, "fixed": 12, "used": 7, "code": 0,
         "ms_auto": 3.0, "ms_fixed": 8.0, "err_auto": 1e-10, "err_fixed": 1e-17, "pass_auto": True,
         "pass_fixed": True},
        {"path": "selector_e2e_summary", "scheme": "I", "tol": 1e-8, "products": 1, "fixed": 12,
         "ms_auto_total": 3.0, "ms_fixed_total": 8.0, "speedup_vs_fixed": 8.0 / 3.0, "pass_auto": 1.0,
         "pass_fixed": 1.0, "mean_used": 7.0},
    ]
    path = tmp_path / "sel.jsonl"
    path.write_text("".join(json.dumps(r) + "\n" for r in rows))
    md = bench.selector_markdown(str(path))
    assert "| I | 1e-08 | 1 | 12 | 7.00 | 100 % | 100 % | 3.0 | 8.0 | 2.67x |" in md
    assert "| I | 2048 | 1.00 | 1e-08 | 7 | 3.00 | 8.00 | 1.00e-10 | 1.00e-17 |" in md


def test_reference_arm_json_line():
    # the reference arm (the oracle, timed on the host's cores) prints the
    # benchmark's JSON line: same metric, unit and config keys as our arm,
    # plus impl, cpu_baseline and a zero-copy e2e
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "512", "--cpu-rows", "8",
                        "--steps", "2", "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["higher_is_better"] is True and line["value"] > 0 and line["unit"] == "TFLOP/s"
    assert line["config"]["n"] == 512 and "workload" in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and "rows" in cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
