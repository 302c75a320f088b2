"""Tolerances of the GPU-vs-oracle parity tests, with their derivations.

The GPU path computes in FP32 (complex64 states, FP32 gate arithmetic); the
oracle in FP64.  On the same Philox draws every difference below is rounding.

TOL_AMP   1e-5 absolute per amplitude: the stated bar.  Measured maximum over
          the shared-prefix, grouped, per-trajectory and fused paths at
          n = 8..24: 2e-7.
TOL_CT    2e-5 absolute per trajectory for <C>_t = sum_x |psi_x|^2 C(x).  Each
          |psi_x|^2 carries a relative FP32 error of at most ~1e-6 after the
          100-300 sweeps of these circuits; C(x) <= E <= 45 edges, and the errors
          of different x have random signs, so the measured maximum is 1.7e-6
          (n = 9..20, every schedule).  TOL_CT is about ten times that.
TOL_MEAN  3e-6 absolute for an ensemble mean <C> against the oracle's mean over
          the same trajectories (a mean of per-trajectory errors: measured at
          most 7e-7).
So a systematic shift of 1e-4 in <C> -- or in any <C>_t -- fails every test
that uses these bounds.
"""
TOL_AMP = 1e-5
TOL_CT = 2e-5
TOL_MEAN = 3e-6
