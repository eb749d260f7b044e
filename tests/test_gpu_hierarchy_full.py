"""The bench workload at full size, in the launch configuration bench.py times:
two detectors x 512 s at 2048 Hz, 2,000 coarse templates at 512 Hz
(N = 2^18) and 20,000 fine templates at 2048 Hz (N = 2^20) filtered on the
neighbourhood union (Sec. III).  One hierarchy step is checked on samples the
FP64 oracle computes one by one (coarse and fine templates, all their
triggers) and, exactly, on the follow-up logic: every followed coarse
template has a coincidence over the ranking threshold, and the stage-2 subset
is the union of the followed templates' neighbourhoods."""

import numpy as np
import pytest

import synth
from oracle import mf_oracle as O
from tests.parity import compare_triggers, oracle_rho2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def test_config2_full_size_sampled(lib):
    from paper_2309_00019_gb300.hierarchy import HierParams, Hierarchy
    from paper_2309_00019_gb300.multi import segment_seed

    c = synth.make_config2(seed=segment_seed(1, 0))  # the bench's segment on rank 0
    hp = HierParams.from_config(c)
    dev = torch.device(DEV)
    h = Hierarchy(hp, c.psd1, c.psd2, len(c.coarse_m1), len(c.fine_m1), c.nbhd_ptr, c.nbhd_idx, device=dev)
    for r0, rows in synth.taylorf2_chunks_torch(c.n1, c.fs1, c.coarse_m1, c.coarse_m2, c.f_low, dev, chunk=256,
                                                ld=h.ld1):
        h.set_bank_rows(1, r0, rows)
    for r0, rows in synth.taylorf2_chunks_torch(c.n2, c.fs2, c.fine_m1, c.fine_m2, c.f_low, dev, chunk=64,
                                                ld=h.ld2):
        h.set_bank_rows(2, r0, rows)
    h.strain.copy_(torch.from_numpy(c.strain))
    n_union = h.run()
    torch.cuda.synchronize()
    trig1, n1, _ = h.p1.triggers()
    trig2, n2, _ = h.p2.triggers()
    co, nco, _ = h.p1.coincs()
    followed = np.nonzero(h.followed.cpu().numpy())[0]
    subset = h.subset[:n_union].cpu().numpy()
    assert n1 == len(trig1) > 0 and n2 == len(trig2) > 0 and len(followed) > 0
    assert nco == len(co)  # every coincidence was stored

    # follow-up logic, exactly: the followed templates are those with a coincidence over the threshold
    # (zero lag or shifted), and the stage-2 subset is the union of their neighbourhoods
    over = co[co["rho_c"] >= c.rho_c_thr]
    assert set(np.unique(over["tmpl"]).tolist()) == set(followed.tolist())
    assert np.array_equal(np.sort(subset), O.nbhd_union(followed, c.nbhd_ptr, c.nbhd_idx))

    s2 = O.strain_to_fd(c.strain.astype(np.float64), c.fs2)
    s1 = O.decimate_fd(s2, c.n1)

    # stage 1: the two coarse templates with the most triggers, a followed one and template 0
    cnt = np.bincount(trig1["tmpl"], minlength=len(c.coarse_m1))
    ids1 = sorted({int(x) for x in np.argsort(-cnt, kind="stable")[:2]} | {int(followed[0]), 0})
    rows1 = synth.taylorf2_torch(c.n1, c.fs1, c.coarse_m1[ids1], c.coarse_m2[ids1], c.f_low, dev).cpu().numpy()
    rho2, _ = oracle_rho2(s1, rows1.astype(np.complex128), c.psd1, c.n1, c.fs1, c.f_low, c.fs1 / 2)
    st1 = compare_triggers(trig1[np.isin(trig1["tmpl"], ids1)], rho2, ids1, c.thr1, c.window1)

    # stage 2: the first, a middle and the last template of the union
    ids2 = sorted({int(subset.min()), int(np.sort(subset)[len(subset) // 2]), int(subset.max())})
    rows2 = synth.taylorf2_torch(c.n2, c.fs2, c.fine_m1[ids2], c.fine_m2[ids2], c.f_low, dev).cpu().numpy()
    rho2, _ = oracle_rho2(s2, rows2.astype(np.complex128), c.psd2, c.n2, c.fs2, c.f_low, c.fs2 / 2)
    st2 = compare_triggers(trig2[np.isin(trig2["tmpl"], ids2)], rho2, ids2, c.thr2, c.window2)
    assert st1["exact"] > 0 and st2["exact"] > 0
    print(f"\nconfig 2 full size: {n1} stage-1 triggers, {nco} coincidences, {len(followed)} followed, "
          f"union {n_union}, {n2} stage-2 triggers; oracle samples: stage 1 {ids1} {st1}, stage 2 {ids2} {st2}")
    h.close()
