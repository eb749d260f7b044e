"""CPU checks of bench.py's host logic: the DRAM-traffic lookup in the committed
profile summaries, the reference arm's JSON line (the oracle timed on the
host) with the keys of the bench contract, and the uneven-length workload's
oracle worker."""

import contextlib
import io
import json
import types

import numpy as np
import pytest

import bench


def test_measured_traffic_reads_and_scales_the_profile_lines():
    full = bench.measured_traffic("k_rows<1024,1024> (stage2)", 128)
    assert full is not None and full > 1e9
    assert bench.measured_traffic("k_rows<1024,1024> (stage2)", 64) == pytest.approx(full / 2)
    assert bench.measured_traffic("k_cols<1024,1024> (stage2)", 128) > 1e9
    assert bench.measured_traffic("k_nothing<1,1> (stage2)", 128) is None


def test_reference_arm_prints_one_contract_line():
    args = types.SimpleNamespace(small=True, steps=1, warmup=0, gpus=1)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.reference_arm(args, 0, 1) == 0
    lines = [l for l in buf.getvalue().splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"]
    # other ranks print nothing
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.reference_arm(args, 1, 2) == 0
    assert buf.getvalue() == ""


def test_uneven_oracle_worker_filters_one_template_over_the_stream():
    import synth

    c = synth.make_config3(seed=2, n_tmpl=6, T=256.0, fs=256.0, f_low=40.0, class_len=(2.0, 8.0), n_inj=1)
    rng = np.random.default_rng(0)
    strain = rng.standard_normal((2, c.n_samples))
    bench._pool_init_uneven(c, strain, 4096)
    td, k, _ = bench._pool_work_uneven((0.0, 0.0, 1, 3))
    assert k == 1 and td == pytest.approx(2 * c.n_samples / c.fs)


def test_fused_kernels_have_no_traffic_until_captured():
    assert bench.measured_traffic("k_cols_h16_fused<1024,1024>", 128) is None
    assert bench.measured_traffic("k_rows_tc_fused<1024,1024>", 128) is None
