"""Two-stage hierarchical search driver (Sec. III) over the libmf C ABI.

Stage 1 filters a coarse bank on the data decimated to the stage-1 rate;
coincident two-detector triggers (zero lag and time-shifted) whose network SNR
passes the follow-up threshold select coarse templates; stage 2 filters the
union of their neighbourhoods in the fine bank at the full rate.  Every step
runs in libmf's kernels on two CUDA streams, stage 1 on its own, ordered by
events (the spectrum before stage 1, the coincidences before the union), so that
the coincidences can be read back while stage 2 runs; PyTorch only provides the
device buffers, the streams and the events.  The host waits once per step, to
size stage 2 from the union count.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import mf


@dataclass
class HierParams:
    n2: int
    fs2: float
    n1: int
    fs1: float
    f_low: float
    thr1: float
    thr2: float
    window1: int
    window2: int
    shift_s: float
    n_shifts: int
    coinc_s: float
    rho_c_thr: float
    n_det: int = 2
    max_trig1: int = 1 << 23
    max_trig2: int = 1 << 25
    max_coincs: int = 1 << 22

    @classmethod
    def from_config(cls, c, **kw):
        return cls(n2=c.n2, fs2=c.fs2, n1=c.n1, fs1=c.fs1, f_low=c.f_low, thr1=c.thr1, thr2=c.thr2,
                   window1=c.window1, window2=c.window2, shift_s=c.shift_s, n_shifts=c.n_shifts,
                   coinc_s=c.coinc_s, rho_c_thr=c.rho_c_thr, **kw)


class Hierarchy:
    """Owns the stage-1 and stage-2 plans and the per-step device buffers."""

    def __init__(self, hp: HierParams, psd1, psd2, n_coarse, n_fine, nbhd_ptr, nbhd_idx, device="cuda:0",
                 stream=None):
        import torch

        self.torch = torch
        self.hp = hp
        self.dev = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.dev)  # the step's stream
        self.stream1 = torch.cuda.Stream(device=self.dev)  # stage 1
        self.ev_fd = torch.cuda.Event()  # the stage-2 spectrum is written
        self.ev_co = torch.cuda.Event()  # stage 1 and its coincidences are done
        self.p2 = mf.Plan(hp.fs2, hp.n2, hp.n_det, hp.f_low, hp.fs2 / 2, hp.thr2, hp.window2,
                          max_triggers=hp.max_trig2, stream=self.stream.cuda_stream)
        self.p1 = mf.Plan(hp.fs1, hp.n1, hp.n_det, hp.f_low, hp.fs1 / 2, hp.thr1, hp.window1,
                          max_triggers=hp.max_trig1, stream=self.stream1.cuda_stream)
        self.p1.set_psd(psd1)
        self.p2.set_psd(psd2)
        self.n_coarse, self.n_fine = n_coarse, n_fine
        self.p1.bank_reserve(n_coarse)
        self.p2.bank_reserve(n_fine)
        self.p2.set_nbhd(nbhd_ptr, nbhd_idx)
        nb1, nb2 = hp.n1 // 2 + 1, hp.n2 // 2 + 1
        self.ld1 = (nb1 + 63) // 64 * 64
        self.ld2 = (nb2 + 63) // 64 * 64
        z = dict(device=self.dev)
        self.strain = torch.zeros((hp.n_det, hp.n2), dtype=torch.float32, **z)
        self.d2 = torch.zeros((hp.n_det, self.ld2), dtype=torch.complex64, **z)
        self.d1 = torch.zeros((hp.n_det, self.ld1), dtype=torch.complex64, **z)
        self.followed = torch.zeros(n_coarse, dtype=torch.int32, **z)
        self.subset = torch.zeros(n_fine, dtype=torch.int32, **z)
        self.n_union = 0
        self.shift1 = int(round(hp.shift_s * hp.fs1))
        self.win1 = int(math.floor(hp.coinc_s * hp.fs1 + 1e-9))

    # -- banks ----------------------------------------------------------------
    def set_bank_rows(self, stage, row0, rows):
        """Copy template rows [row0, row0+len) of the stage-1 (stage=1) or stage-2
        bank from a host array or device tensor [rows, >= N/2+1] (complex64)."""
        plan, ld = (self.p1, self.ld1) if stage == 1 else (self.p2, self.ld2)
        if isinstance(rows, np.ndarray):
            rows = np.ascontiguousarray(rows, dtype=np.complex64)
            plan.bank_set_rows(row0, rows, on_device=0)
        else:
            plan.bank_set_rows(row0, rows, on_device=1)

    # -- one step ---------------------------------------------------------------
    def _stage1(self, s):
        """Spectrum (step stream), stage 1 and coincidences (stage-1 stream), union (step stream, waits)."""
        hp = self.hp
        self.p2.strain_to_fd(s, self.d2, ld_strain=hp.n2, ld_dtilde=self.ld2)
        self.ev_fd.record(self.stream)
        self.stream1.wait_event(self.ev_fd)
        self.p1.decimate(self.d2, self.d1, ld_in=self.ld2, ld_out=self.ld1)
        self.p1.filter(self.d1, ld=self.ld1)
        self.p1.coincide(self.followed, self.shift1, hp.n_shifts, self.win1, hp.rho_c_thr,
                         max_coincs=hp.max_coincs)
        self.ev_co.record(self.stream1)
        self.stream.wait_event(self.ev_co)
        self.n_union = self.p2.nbhd_union(self.followed, self.subset)

    def run(self, strain=None):
        """Whole hot path on device-resident strain [n_det, n2] (default: self.strain); every step of it is
        ordered on the step's stream (self.stream) by its end."""
        self._stage1(self.strain if strain is None else strain)
        self.p2.filter(self.d2, subset=self.subset, n_subset=self.n_union, ld=self.ld2)
        return self.n_union

    def run_host(self, strain_host):
        """End to end from host strain (pinned for an asynchronous copy): H2D, the
        whole hot path, and D2H of the stage-2 triggers and stage-1 coincidences into
        page-locked buffers of the plans (the returned arrays are overwritten by the
        next call)."""
        with self.torch.cuda.stream(self.stream):
            self.strain.copy_(strain_host, non_blocking=True)
        self.run()
        # stage 1's stream is idle by now: its coincidences are read (and ordered on the host) while stage 2 runs
        co, nco, _ = self.p1.coincs(pinned=True)
        trig2, n2, _ = self.p2.triggers(pinned=True)  # page-locked readback, valid until the next step
        return trig2, co

    def td_seconds(self):
        """Template-seconds filtered by the last step (both stages, every detector)."""
        hp = self.hp
        t1 = self.n_coarse * hp.n_det * hp.n1 / hp.fs1
        t2 = self.n_union * hp.n_det * hp.n2 / hp.fs2
        return t1 + t2

    def close(self):
        self.p1.close()
        self.p2.close()
