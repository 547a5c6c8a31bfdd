"""Host-side pieces of bench.py's JSON line: the roofline object for each kind of
headline (FP64 sweep against the FP64 pipe; the two-step FP32 form with its
measured DRAM bytes and per-launch traffic; one step per launch against HBM) and
the launch count of the two-step form."""
import argparse

import bench


def _args(**kw):
    a = dict(compute="f64", storage="f64", workload="mms", shift="auto", sweep="auto", steps=1000, n=8192)
    a.update(kw)
    return argparse.Namespace(**a)


def test_fp64_roofline_is_the_fp64_pipe():
    nodes, t = 8192 * 8192, 6.46e-3
    peak = {"tops": 0.6, "by_kind_tops": {"fma": 0.6, "add": 0.6, "mul": 0.6}, "mix": bench.FP64_MIX_PER_UPDATE,
            "kernel": "probe"}
    r = bench.roofline(_args(), nodes, t, 160 * nodes / t / 1e9, 6800.0, "measured", peak)
    assert r["bound"] == "alu" and r["unit"] == "T FP64 op/s"
    assert r["ops_per_update"] == bench.FP64_OPS_PER_UPDATE_LINEAR
    assert abs(r["achieved"] - bench.FP64_OPS_PER_UPDATE_LINEAR * nodes / t / 1e12) < 1e-3
    # the measured rate is the peak; the nominal one is reported beside it
    assert r["peak"] == 0.6 and "measured" in r["peak_kind"]
    assert abs(r["frac"] - r["achieved"] / 0.6) < 1e-3
    assert abs(r["frac_of_nominal"] - r["achieved"] / bench.FP64_NOMINAL_TOPS) < 1e-3
    assert r["traffic"] == round(bench.FP64_TRAFFIC_PER_NODE * nodes)
    assert r["hbm_view"]["bytes_per_update"] == 160
    # without a measurement the nominal rate is used and said so
    r0 = bench.roofline(_args(), nodes, t, 1.0, 6800.0, "measured")
    assert r0["peak"] == bench.FP64_NOMINAL_TOPS and "not measured" in r0["peak_kind"]


def test_fp64_operation_count_belongs_to_the_current_kernel():
    """The FP64 operation count (kept next to collide_fold) and the ncu capture of
    the FP64 sweep were taken for the kernel sources with FP64_SWEEP_DIGEST.  An
    edit to those sources fails here until the count is re-checked, the capture
    re-taken and the digest updated, so the roofline cannot go stale silently."""
    assert bench.source_digest(bench.FP64_SWEEP_SOURCES) == bench.FP64_SWEEP_DIGEST, (
        "FP64 sweep sources changed: recount kFp64OpsPerNodeLinearTrig, recapture the FP64 sweep "
        "with ncu, then update FP64_SWEEP_DIGEST / FP64_TRAFFIC_PER_NODE")
    assert bench.FP64_OPS_PER_UPDATE_LINEAR == 50 == sum(bench.FP64_MIX_PER_UPDATE.values())


def test_stale_captures_are_reported_as_null(monkeypatch):
    nodes, t = 4096 * 4096, 1e-3
    monkeypatch.setattr(bench, "FP64_SWEEP_DIGEST", "0" * 16)
    assert bench.roofline(_args(), nodes, t, 1.0, 6800.0, "measured")["traffic"] is None
    monkeypatch.setattr(bench, "TB2_DIGEST", "0" * 16)
    r = bench.roofline(_args(compute="f32", storage="f32", shift="ref"), nodes, t, 1.0, 6800.0, "measured")
    assert r["traffic"] is None and r["dram_bytes_per_update"] is None


def test_two_step_roofline_reports_measured_dram_bytes(monkeypatch):
    # as if the capture were of the current two-step sources
    monkeypatch.setattr(bench, "TB2_DIGEST", bench.source_digest(bench.TB2_SOURCES))
    nodes, t = 8192 * 8192, 0.536e-3
    args = _args(compute="f32", storage="f32", shift="ref")
    assert bench.two_step_form(args)
    r = bench.roofline(args, nodes, t, 80 * nodes / t / 1e9, 6800.0, "measured")
    assert r["bound"] == "hbm" and r["kernel"].startswith("sweep_tb2_kernel")
    assert r["dram_bytes_per_update"] == bench.TB2_DRAM_BYTES_PER_UPDATE[("f32", "ref")]
    assert r["traffic"] == round(r["dram_bytes_per_update"] * 2 * nodes)   # one launch = two steps
    assert r["frac"] > 1.0   # algorithmic one-step bytes over the copy peak
    # the local shift is the default for 16-bit storage (two-step form asked for)
    r16 = bench.roofline(_args(compute="f32", storage="f16", sweep="tb2"), nodes, t, 1.0, 6800.0, "measured")
    assert r16["dram_bytes_per_update"] == bench.TB2_DRAM_BYTES_PER_UPDATE[("f16", "local")]


def test_auto_kernel_form_follows_the_library():
    """AUTO resolves as the library does: the vector form for FP16/BF16 storage on
    large lattices, two steps per launch for FP32 storage and small lattices, the
    plain sweep for FP64 and double-word."""
    assert bench.kernel_form(_args(compute="f32", storage="f16")) == "vec"
    assert bench.kernel_form(_args(compute="f32", storage="bf16")) == "vec"
    assert bench.kernel_form(_args(compute="f32", storage="f32")) == "tb2"
    assert bench.kernel_form(_args(compute="f32", storage="f16", workload="nonlinear")) == "vec"
    assert bench.two_step_form(_args(compute="f32", storage="f16", sweep="tb2v"))
    assert bench.kernel_form(_args(compute="f32", storage="f16", n=1024)) == "tb2"   # small: fewer launches
    assert bench.kernel_form(_args()) == "plain"
    assert bench.kernel_form(_args(compute="df64", storage="df64")) == "plain"
    assert bench.kernel_form(_args(compute="f32", storage="f16", sweep="plain")) == "plain"
    r = bench.roofline(_args(compute="f32", storage="f16"), 4096 * 4096, 1e-3, 6000.0, 6800.0, "measured")
    assert r["bound"] == "hbm" and r["kernel"].startswith("sweep_vec_kernel") and r["bytes_per_update"] == 44


def test_one_step_forms_and_launch_counts():
    nodes = 4096 * 4096
    args = _args(compute="f32", storage="f32", shift="ref", sweep="plain")
    assert not bench.two_step_form(args)
    r = bench.roofline(args, nodes, 1e-3, 6000.0, 6800.0, "measured")
    assert r["kernel"].startswith("sweep_kernel") and r["traffic"] is None
    assert not bench.two_step_form(_args())                       # FP64: one launch per step
    assert not bench.two_step_form(_args(compute="df64", storage="df64"))
