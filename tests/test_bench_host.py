"""Host-side logic of bench.py: workload bookkeeping, the whole-job value,
max-over-ranks timing on a 2-rank gloo group (the multi-GPU path is
replicas only), clock-sample parsing and the reference (CPU oracle) arm."""
import json
import os
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_op_list_is_the_sweep():
    ops = bench.op_list()
    assert len(ops) == 18
    assert len({o[0] for o in ops}) == 18
    kinds = [o[1] for o in ops]
    assert kinds.count("gemv") == 12 and kinds.count("dot") == 2 and kinds.count("ger") == 4


@pytest.mark.parametrize("kind,dt,m,n,want", [
    ("gemv", "f64", 4096, 4096, 134_316_032),
    ("gemv", "f32", 16384, 16384, 1_073_938_432),
    ("gemv", "f64", 16384, 16384, 2_147_876_864),
    ("gemv", "f32", 1048576, 64, 276_824_320),
    ("gemv", "f64", 1048576, 64, 553_648_640),
    ("gemv", "f32", 64, 1048576, 272_630_272),
    ("gemv", "f64", 64, 1048576, 545_260_544),
    ("ger", "f32", 16384, 16384, 2_147_614_720),
    ("ger", "f64", 16384, 16384, 4_295_229_440),
    ("dot", "f64", 1, 1 << 28, 8 * (2 * (1 << 28) + 2)),
])
def test_algorithmic_bytes(kind, dt, m, n, want):
    assert bench.alg_bytes(kind, dt, m, n) == want


def test_whole_job_value():
    assert bench.whole_job_value(1e9, 10, 1, 2.0) == pytest.approx(5.0)
    assert bench.whole_job_value(1e9, 10, 4, 2.0) == pytest.approx(20.0)


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench as b
    w, r = b.init_dist("gloo")
    b.barrier()
    mx = b.max_over_ranks(1.5 + r)
    out.put((r, w, mx))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2, 2.5), (1, 2, 2.5)]


def test_clock_summary_parsing():
    cs = bench.ClockSampler(0)
    row = lambda mhz, pc: ["2026/01/01", str(mhz), "2070", "900", "0x0", "Not Active",
                           "Not Active", "Not Active", pc]
    cs.samples = [(10.0, row(1900, "Not Active")), (11.0, row(1950, "Active")),
                  (12.0, row(2000, "Not Active")), (13.0, row(1000, "Not Active"))]
    s = cs.summary(9.5, 12.5)
    assert s["sm_mhz"] == 1950 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3


def test_reference_arm_prints_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "impl", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "cpu_baseline", "e2e", "config"):
        assert k in line, k
    assert line["impl"] == "reference" and line["unit"] == "GB/s" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_source_sha_ignores_comments_only():
    import bench
    a = "int f(int x) {  // twice\n  return 2 * x; /* doubled */\n}\n"
    b = "/* header */\nint f(int x) {\n\n  return 2 * x;\n}  // end\n"
    c = "int f(int x) { return 3 * x; }"
    assert bench.code_of(a) == bench.code_of(b) != bench.code_of(c)


def test_link_bound():
    """The e2e step bound: the slowest of upload alone, download alone and
    both directions at their shared rate (figures of a GB300 machine)."""
    link = {"h2d_GB_s": 210.7, "d2h_GB_s": 193.0, "both_GB_s": 299.2}
    b = bench.link_bound(29.07e9, 17.74e9, 6.455e9, link)
    assert abs(b - 29.07e9 / (17.74e9 / 210.7e9) / 1e9) < 1e-6        # the upload decides
    assert abs(b - 345.3) < 0.5
    up_only = bench.link_bound(10e9, 10e9, 0, link)
    assert abs(up_only - 210.7) < 1e-9
    both = bench.link_bound(10e9, 5e9, 5e9, {"h2d_GB_s": 100.0, "d2h_GB_s": 100.0, "both_GB_s": 100.0})
    assert abs(both - 100.0) < 1e-9                                     # the shared rate decides


def test_fit_fixed_cost_recovers_a_line():
    """t = t0 + bytes / bw is recovered exactly from points on the line, and
    least squares splits symmetric noise evenly; fewer than two distinct
    sizes give no fit."""
    t0, bw = 6e-6, 7.3e12
    pts = [(k * 272_630_272, t0 + k * 272_630_272 / bw) for k in (1, 2, 4, 8)]
    f0, fbw = bench.fit_fixed_cost(pts)
    assert abs(f0 - t0) < 1e-12 and abs(fbw / bw - 1) < 1e-9
    noisy = [(b, t + (1e-7 if i % 2 else -1e-7)) for i, (b, t) in enumerate(pts)]
    g0, gbw = bench.fit_fixed_cost(noisy)
    assert abs(g0 - t0) < 2e-7 and abs(gbw / bw - 1) < 1e-2
    assert bench.fit_fixed_cost(pts[:1]) == (None, None)
    assert bench.fit_fixed_cost([pts[0], pts[0]]) == (None, None)
    assert bench.fit_fixed_cost([(1.0, 2.0), (2.0, 1.0)])[1] is None   # falling time: no rate


def test_roofline_of_picks_the_binding_resource():
    """GER moves 16 bytes per 2 flops, so even FP64 GER is bound by HBM; a
    FP64 GEMV's 2 flops per 8 bytes would outrun the FP64 pipe's nominal
    2 FMA/clk/SM, so its roofline is the ALU one (the kernels take most of
    those products off that pipe, which is why they can beat it)."""
    hbm = 6697.8
    ger = ("ger_row_f64", "ger", "f64", "row", 16384, 16384)
    by = bench.alg_bytes("ger", "f64", 16384, 16384)
    r = bench.roofline_of(ger, by / (6000.0 * 1e9), hbm, "measured")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 6000.0) < 0.1 and abs(r["frac"] - 6000.0 / hbm) < 1e-4
    assert r["algorithmic_bytes"] == by
    traffic = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))["kernels"]["ger_row_f64"]
    want = traffic["dram_bytes_per_launch"] if traffic["sha"] == bench.source_sha(traffic["sources"]) else None
    assert r["traffic"] == want
    gemv = ("gemv_row_sq_f64", "gemv", "f64", "row", 16384, 16384)
    flops = bench.alg_flops("gemv", 16384, 16384)
    r = bench.roofline_of(gemv, flops / 1.0e12, hbm, "measured")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    peak = bench.SMS * bench.DP_FMA_PER_CLK_SM * 2 * bench.SM_MAX_MHZ * 1e6 / 1e12
    assert abs(r["peak"] - peak) < 1e-3 and abs(r["achieved"] - 1.0) < 1e-3
    f32 = ("gemv_row_sq_f32", "gemv", "f32", "row", 16384, 16384)
    assert bench.roofline_of(f32, 1e-4, hbm, "measured")["bound"] == "hbm"   # FP32 has no ALU leg
