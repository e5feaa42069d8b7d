"""awo_simulate_time_kernel: the events it hands over bracket the particle
kernel of the next awo_simulate call alone, are consumed by that call, and
change nothing in its results."""
import numpy as np
import pytest
import torch

import paper_2506_23364_gb300 as awo
from paper_2506_23364_gb300 import inputs

pytestmark = pytest.mark.gpu


def _events(k):
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
    for e in evs:  # torch creates an event at its first record
        e.record()
    torch.cuda.synchronize()
    return evs


def _overlay():
    w = inputs.tiny()
    ov = awo.Overlay(w.width, w.height, w.cell_size, quantised=False, levels=1)
    ov.load_dem(w.dem_f32)
    ov.terrain(w.slope_lo_deg, w.slope_hi_deg)
    return w, ov


def test_events_bracket_the_particle_kernel_only():
    w, ov = _overlay()
    p = awo.SimParams.make(traj_per_cell=w.traj_per_cell, max_steps=w.max_steps, seed=5)
    ov.simulate(p)
    torch.cuda.synchronize()
    ref = (ov.count.cpu().numpy().copy(), ov.maxe.cpu().numpy().copy(), ov.stats_dict())
    assert ref[2]["total_steps"] > 0

    k0, k1, c0, c1 = _events(4)
    c0.record()
    awo.awo_simulate_time_kernel(k0, k1)
    ov.simulate(p)
    c1.record()
    torch.cuda.synchronize()
    kernel_ms, call_ms = k0.elapsed_time(k1), c0.elapsed_time(c1)
    assert 0.0 < kernel_ms <= call_ms
    assert np.array_equal(ov.count.cpu().numpy(), ref[0])
    assert np.array_equal(ov.maxe.cpu().numpy(), ref[1])
    assert ov.stats_dict() == ref[2]

    # consumed: a later call without the hook leaves both events where they were
    ov.simulate(p)
    torch.cuda.synchronize()
    assert k0.elapsed_time(k1) == kernel_ms


def test_withdrawn_events_are_not_recorded():
    w, ov = _overlay()
    p = awo.SimParams.make(traj_per_cell=4, max_steps=w.max_steps, seed=1)
    k0, k1 = _events(2)
    before = k0.elapsed_time(k1)
    awo.awo_simulate_time_kernel(k0, k1)
    awo.awo_simulate_time_kernel(None, None)
    ov.simulate(p)
    torch.cuda.synchronize()
    assert k0.elapsed_time(k1) == before


def test_no_particle_kernel_gives_an_empty_interval():
    """max_steps = 0: the prologue alone runs (every particle capped at its
    release visit) and both events are recorded after it."""
    w, ov = _overlay()
    p = awo.SimParams.make(traj_per_cell=4, max_steps=0, seed=1)
    k0, k1, c0, c1 = _events(4)
    c0.record()
    awo.awo_simulate_time_kernel(k0, k1)
    ov.simulate(p)
    c1.record()
    torch.cuda.synchronize()
    assert 0.0 <= k0.elapsed_time(k1) <= c0.elapsed_time(c1)
    st = ov.stats_dict()
    assert st["total_steps"] == 0 and st["n_traj"] == st["n_capped"] == 4 * ov.n_release()
