"""GPU parity of the whole two-stage hot path (Sec. III) against the oracle's
own two-stage run on the same seeded inputs: stage-1 triggers, time-shifted
coincidences, follow-up set, neighbourhood union and stage-2 triggers."""

import numpy as np
import pytest

import synth
from oracle import mf_oracle as O
from tests.parity import compare_triggers, oracle_rho2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small_run(lib):
    from paper_2309_00019_gb300.hierarchy import HierParams, Hierarchy

    c = synth.make_config2(small=True)
    coarse = c.coarse_bank()
    fine = c.fine_bank()
    h = Hierarchy(HierParams.from_config(c), c.psd1, c.psd2, len(coarse), len(fine), c.nbhd_ptr, c.nbhd_idx)
    h.set_bank_rows(1, 0, coarse)
    h.set_bank_rows(2, 0, fine)
    h.strain.copy_(torch.from_numpy(c.strain))
    n_union = h.run()
    torch.cuda.synchronize()
    ref = O.hierarchical_search(c.strain, c.fs2, c.n2, c.fs1, c.psd1, c.psd2, coarse.astype(np.complex128),
                                fine.astype(np.complex128), c.nbhd_ptr, c.nbhd_idx, c.f_low, c.thr1, c.thr2,
                                c.window1, c.window2, c.shift_s, c.n_shifts, c.coinc_s, c.rho_c_thr)
    return dict(c=c, h=h, n_union=n_union, ref=ref, coarse=coarse, fine=fine)


def test_stage1_triggers(small_run):
    c, h, ref = small_run["c"], small_run["h"], small_run["ref"]
    trig1, n1, _ = h.p1.triggers()
    rho2, _ = oracle_rho2(ref["stilde1"], small_run["coarse"], c.psd1, c.n1, c.fs1, c.f_low, c.fs1 / 2)
    st = compare_triggers(trig1, rho2, range(len(small_run["coarse"])), c.thr1, c.window1)
    assert st["exact"] == n1 == len(ref["trig1"])


def test_coincidences_followup_and_union(small_run):
    c, h, ref = small_run["c"], small_run["h"], small_run["ref"]
    co, nco, _ = h.p1.coincs()
    want = ref["coinc"][ref["coinc"]["rho_c"] >= c.rho_c_thr]
    got_keys = [(int(x["tmpl"]), int(x["shift"]), int(x["sample0"]), int(x["sample1"])) for x in co]
    want_keys = [(int(x["tmpl"]), int(x["shift"]), int(x["sample0"]), int(x["sample1"])) for x in want]
    assert got_keys == want_keys and nco > 0
    assert np.allclose(co["rho_c"], want["rho_c"], rtol=1e-4)
    # a read into a smaller buffer: the first records of the same order, and the overflow status
    from paper_2309_00019_gb300 import mf
    if nco > 3:
        co3, n3, st3 = h.p1.coincs(cap=3)
        assert n3 == nco and st3 == mf.MF_EOVERFLOW
        assert [(int(x["tmpl"]), int(x["shift"]), int(x["sample0"]), int(x["sample1"])) for x in co3] == got_keys[:3]
    assert np.any(co["shift"] == 0) and np.any(co["shift"] > 0)  # zero-lag and time-shifted follow-ups
    followed = np.nonzero(h.followed.cpu().numpy())[0]
    assert list(followed) == list(ref["followed"])
    assert small_run["n_union"] == len(ref["union"])
    assert list(h.subset[: small_run["n_union"]].cpu().numpy()) == list(ref["union"])


def test_stage2_triggers(small_run):
    c, h, ref = small_run["c"], small_run["h"], small_run["ref"]
    trig2, n2, _ = h.p2.triggers()
    union = ref["union"]
    rho2, _ = oracle_rho2(ref["stilde2"], small_run["fine"][union], c.psd2, c.n2, c.fs2, c.f_low, c.fs2 / 2)
    st = compare_triggers(trig2, rho2, union, c.thr2, c.window2)
    assert st["exact"] == n2 == len(ref["trig2"])
    assert h.td_seconds() == pytest.approx(len(small_run["coarse"]) * 2 * 32 + len(union) * 2 * 32)


def test_end_to_end_from_host_strain(small_run):
    c, h = small_run["c"], small_run["h"]
    pinned = torch.from_numpy(c.strain).pin_memory()
    trig2, co = h.run_host(pinned)
    trig_dev, _, _ = h.p2.triggers()
    assert np.array_equal(trig2, trig_dev)
    assert len(co) > 0
    # a second pinned read reuses the plan's page-locked buffer and gives the same records
    again, _, _ = h.p2.triggers(pinned=True)
    assert np.array_equal(again, trig_dev)


def test_background_far_of_the_coincidences(small_run):
    """Eq. (6) and the Sec. IV tail fit through mf_far on the run's own
    coincidences (zero lag = foreground, shifted = background) against the oracle."""
    from paper_2309_00019_gb300 import mf

    c, h = small_run["c"], small_run["h"]
    co, _, _ = h.p1.coincs()
    fg = co["rho_c"][co["shift"] == 0]
    bg = co["rho_c"][co["shift"] > 0]
    assert len(fg) > 0 and len(bg) > 2
    t_bg = c.n_shifts * (c.n1 / c.fs1)
    fit_min = float(np.sort(bg)[len(bg) // 3])
    fc, ff, a, b = mf.far(fg, bg, t_bg, scale=3.0, fit_min=fit_min)
    fg64, bg64 = fg.astype(np.float64), bg.astype(np.float64)
    assert np.array_equal(fc, O.far_count(fg64, bg64, t_bg, scale=3.0))
    ra, rb = O.tail_fit(bg64, fit_min, scale=3.0)
    assert a == pytest.approx(ra, rel=1e-9, abs=1e-9) and b == pytest.approx(rb, rel=1e-9, abs=1e-9)
    assert np.allclose(ff, O.far_fit(fg64, ra, rb, t_bg), rtol=1e-9)


def test_far_edge_cases(lib):
    from paper_2309_00019_gb300 import mf

    fc, ff, a, b = mf.far([8.0, 9.0], [7.0], 10.0, fit_min=5.0)
    assert np.allclose(fc, [0.1, 0.1]) and np.isnan(a) and np.all(np.isnan(ff))  # one value: no fit
    fc, ff, a, b = mf.far([7.0], [7.0, 7.0, 8.0], 2.0, fit_min=7.0)
    assert fc[0] == pytest.approx(2.0)  # (1 + 3) / 2: ties count
    with pytest.raises(mf.MFError):
        mf.far([1.0], [1.0], 0.0)
