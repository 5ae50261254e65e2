"""bench.py's host-side legs on the CPU: the oracle samples timed beside the
factorised and continuous steps run on a small workload and return a
positive time with a description of the sample."""
import math

import numpy as np

import bench
from synth import continuous_maps, workload


def test_cpu_legs_small_workload():
    w = workload("periodic32", scale=0.2)
    pa = np.zeros((18, 36))
    pa[12:, :] = 1.0 / (2.0 * math.pi * (1.0 - math.sin(math.radians(30.0))))
    sel = dict(n_tot=float(w["data"].n), p_ang=pa, p_z=np.full(4, 1.0 / 0.04), z_lo=0.02, z_hi=0.06, z_max=0.07,
               h0=100.0, omega_m=0.307, omega_k=0.0, omega_l=0.693, c=300000.0)
    ms, sample = bench.cpu_oracle_mode_sample(w, (2, 3), "factorised", selection=sel, cells=200)
    assert ms > 0 and "Eq. 7" in sample
    D, R = continuous_maps(1, (32, 32, 32), 10.0)
    ms, sample = bench.cpu_oracle_mode_sample(w, (2, 3), "continuous", maps=(D, R))
    assert ms > 0 and "Eq. 15" in sample
