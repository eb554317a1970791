"""Measurement helpers of bench.py (CPU): the Mie series used for the error of
the large solve agrees with the oracle's, and the committed ncu summary of the
FP32 far kernel still describes the current source (its DRAM traffic is used)."""
import numpy as np

import bench
import oracle


def test_bench_mie_series_matches_oracle():
    rng = np.random.default_rng(3)
    pts = rng.normal(size=(50, 3))
    pts /= np.linalg.norm(pts, axis=1, keepdims=True)
    for k, d in ((5.0, (0.0, 0.0, 1.0)), (16.0, (1.0, 2.0, -0.5))):
        a = bench.mie_density_sphere(k, d, pts)
        b = oracle.mie_density(k, d, pts)
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


def test_far_profile_matches_source():
    assert bench.far_traffic_per_launch() is not None


def test_bench_mie_scattered_field_cancels_the_incident_wave_on_the_sphere():
    """Sound-soft boundary: p_inc + p_sca = 0 on the unit sphere."""
    rng = np.random.default_rng(5)
    pts = rng.normal(size=(40, 3))
    pts /= np.linalg.norm(pts, axis=1, keepdims=True)
    for k, d in ((5.0, np.array([0.0, 0.0, 1.0])), (16.0, np.array([1.0, 0.0, 0.0]))):
        s = bench.mie_scattered_sphere(k, d, pts)
        assert np.max(np.abs(s + np.exp(1j * k * pts @ d))) < 1e-9


def test_bench_pec_mie_matches_the_oracle():
    import bench
    import oracle
    mu = np.cos(np.linspace(0.05, np.pi - 0.05, 9))
    for k in (1.0, 8.0):
        a1, a2 = bench.mie_pec_sphere(k, mu)
        b1, b2 = oracle.mie_pec_amplitudes(k, mu)
        assert np.abs(a1 - b1).max() < 1e-12 * np.abs(b1).max() and np.abs(a2 - b2).max() < 1e-12 * np.abs(b2).max()


def test_clock_sampler_parses_nvidia_smi_lines(tmp_path):
    """The clocks record of a bench line: median SM clock, maximum clock and power,
    throttle reasons that were active, from nvidia-smi's CSV lines (a stand-in
    process replaces nvidia-smi)."""
    import os
    cs = bench.ClockSampler("0")
    cs.path = str(tmp_path / "clocks.csv")
    with open(cs.path, "w") as f:
        f.write("0, 2070 MHz, 2070 MHz, 500.12 W, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 1980 MHz, 2070 MHz, 900.00 W, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n")
        f.write("garbage line\n")

    class Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

        def kill(self):
            pass

    cs.proc = Proc()
    cs.fh = open(os.devnull, "w")
    out = cs.stop()
    assert out["samples"] == 2 and out["sm_mhz"] == 2025.0 and out["sm_max_mhz"] == 2070.0
    assert out["power_w_max"] == 900.0 and out["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(cs.path)
