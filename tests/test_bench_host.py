"""Host legs of bench.py on CPU: the oracle split over host threads by environment range
does the same work, and gives the same states, as one unsharded call."""
import types
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import bench
import oracle
from paper_2606_08039_gb300 import workloads as wl


def _args(**kw):
    a = dict(model="cf2x", integrator="euler", gnd_heights="com", actions="pid", controller="pid",
             randomize=False)
    a.update(kw)
    return types.SimpleNamespace(**a)


@pytest.mark.parametrize("kw", [{}, {"controller": "dsl"}, {"actions": "mixed"}])
def test_sharded_oracle_equals_one_call(kw):
    args = _args(**kw)
    sw = wl.full_aero(1, n_envs=24)
    one = bench.OracleShards(args, sw, 1, 1)
    many = bench.OracleShards(args, sw, 1, 5)
    assert len(many.shards) == 5
    assert sum(sh["x"].shape[0] for sh in many.shards) == sw.n
    with ThreadPoolExecutor(5) as pool:
        for _ in range(2):
            one.step(None)
            many.step(pool)
    x_many = np.concatenate([sh["x"] for sh in many.shards])
    np.testing.assert_array_equal(one.shards[0]["x"], x_many)
    np.testing.assert_array_equal(one.shards[0]["integ"], np.concatenate([sh["integ"] for sh in many.shards]))


def test_sharded_oracle_under_randomization_keeps_each_environments_row():
    args = _args(randomize=True)
    sw = wl.full_aero(1, n_envs=10)
    many = bench.OracleShards(args, sw, 1, 3)
    _, _, _, dr = bench.oracle_workload(args, sw, 1)
    rows = np.concatenate([sh["dr"].env_dr for sh in many.shards])
    np.testing.assert_array_equal(rows, dr.env_dr)
    many.step(None)
    for sh in many.shards:
        assert np.isfinite(sh["x"]).all()


def test_more_threads_than_environments():
    sw = wl.full_aero(1, n_envs=3)
    sh = bench.OracleShards(_args(), sw, 1, 8)
    assert len(sh.shards) == 3
    assert bench.host_cores() >= 1


def test_reference_arm_prints_nothing_on_other_ranks(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(_args(steps=1, warmup=3, gpus=2))
    assert capsys.readouterr().out == ""


def test_in_place_oracle_call_equals_the_wrapper():
    """oracle.control_steps_into (no copies, used for timing) gives control_steps' results."""
    args = _args()
    sw = wl.full_aero(1, n_envs=12)
    sh = bench.OracleShards(args, sw, 1, 1)
    acts, wp, sp, dr = bench.oracle_workload(args, sw, 1)
    x0 = sw.x13().astype(np.float64)
    x, integ, a, kin, nbr_i, nbr_r = oracle.control_steps(sh.P, sw.env_off, sw.flags.astype(np.int32), acts, x0,
                                                          np.zeros((sw.n, 6)), np.zeros((sw.n, 4)), wp, 5, obs=True)
    sh.step(None)
    s0 = sh.shards[0]
    np.testing.assert_array_equal(s0["x"], x)
    np.testing.assert_array_equal(s0["integ"], integ)
    np.testing.assert_array_equal(s0["kin"], kin)
    np.testing.assert_array_equal(s0["idx"], nbr_i)
    np.testing.assert_array_equal(s0["rel"], nbr_r)


def test_clock_summary_uses_the_samples_inside_the_timed_region():
    """ClockSampler.stop(windows): the median and the throttle reasons come from the samples
    read inside the timed windows (falling back to every sample when none is inside)."""
    cs = bench.ClockSampler(0)

    class _Done:  # a finished sampler process
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    class _Joined:
        def join(self, timeout=None):
            pass

    idle = "0, 1200, 2070, 150.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    load = "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Active"
    cs.proc, cs.thread = _Done(), _Joined()
    cs.lines = [(0.0, idle), (1.0, load), (1.1, load), (2.0, idle)]
    inside = cs.stop(windows=[(0.95, 1.15)])
    assert inside["sm_mhz"] == 2070 and inside["samples"] == 2 and inside["window"] == "timed region"
    assert inside["reasons"] == ["sw_power_cap"]
    cs.proc, cs.thread = _Done(), _Joined()
    everything = cs.stop(windows=[(5.0, 6.0)])
    assert everything["samples"] == 4 and everything["window"] == "whole run"


def test_algorithmic_bytes_per_drone_and_control_step():
    """The bytes the roofline divides by: 360 B per drone for PID waypoints (the 13-value state
    and the 6 integrals read and written, the waypoint, KIN + indices + features), 312 B for
    plain RPM actions (no integrals), +32 B with the DSL setpoint, and 520 B under
    randomization with an action history of depth 3 (rotor speeds, history shift, the row and
    wind state of each four-drone environment)."""
    sw = wl.full_aero(1, n_envs=64)
    n = sw.n
    pid = np.full(sw.n_envs, 1, np.uint8)
    rpm = np.zeros(sw.n_envs, np.uint8)
    assert bench.algorithmic_bytes(sw, pid, 1, False) == 360 * n
    assert bench.algorithmic_bytes(sw, rpm, 0, False) == 312 * n
    assert bench.algorithmic_bytes(sw, pid, 1, True) == 392 * n
    assert bench.algorithmic_bytes(sw, pid, 1, False, dr_depth=3) == 520 * n
    assert bench.BYTES_PER_DRONE_STEP == 360


def test_binding_roofline_takes_the_longer_ideal_time():
    peaks = {"hbm_gbs": 1000.0, "src": "test"}
    # 1 GB at 1000 GB/s is 1 ms; a tiny flop count: HBM binds
    r = bench.binding_roofline(1e9, 1e6, 2e-3, peaks)
    assert r["bound"] == "hbm" and r["achieved"] == pytest.approx(500.0) and r["frac"] == pytest.approx(0.5)
    assert r["other_bound"]["bound"] == "alu"
    # many flops, few bytes: the ALU binds
    r = bench.binding_roofline(1e3, bench.FP32_PEAK_TFLOPS * 1e12 * 1e-3, 4e-3, peaks)
    assert r["bound"] == "alu" and r["frac"] == pytest.approx(0.25)
