"""Comparison rules between the CUDA path and the FP64 oracle.

Tolerances (the planner's accuracy targets):
* per-sample cost S: |S_gpu - S_oracle| <= 1e-4 * max(|S_oracle|, 1), for every sample;
* updated controls u* and the optimal trajectory x*: 1e-4 absolute, always (they do
  not depend on which sample of a near tie is the argmin: the shift by S_min cancels
  between the numerator and the normaliser of Eq. (11));
* Philox words: bit-exact; argmin index: exact unless the oracle's two lowest
  costs are within 1e-4 relative (a near tie), where the GPU's index must lie in
  the oracle's near-tie set.

The step cost has jumps (the reference yaw switches between polyline segments,
c_target's indicator, the collision-only switch, the yaw wrap).  The oracle
reports, per sample, how far (metres / radians) the rollout passed from the
nearest jump.  A sample whose margin is below MARGIN_EXCUSE may land on the other
side of a jump in binary32; such a sample may miss the cost tolerance only if it
is one of at most MAX_EXCUSED_FAIL of the samples (0.1 %), and every sample farther
from a jump must meet it.  A test that allows excused misses says so explicitly.
"""
import numpy as np

S_REL_TOL = 1e-4
U_ABS_TOL = 1e-4
X_ABS_TOL = 1e-4
MARGIN_EXCUSE = 1e-5
MAX_EXCUSED_FAIL = 1e-3
NEAR_TIE = 1e-4


def cost_report(S_gpu, S_orc, margin):
    rel = np.abs(S_gpu - S_orc) / np.maximum(np.abs(S_orc), 1.0)
    excused = margin < MARGIN_EXCUSE
    over = rel > S_REL_TOL
    bad = over & ~excused
    return dict(max_rel=float(rel[~excused].max()) if (~excused).any() else 0.0,
                max_rel_all=float(rel.max()) if rel.size else 0.0,
                excused=int(excused.sum()), frac_excused=float(excused.mean()) if rel.size else 0.0,
                n_bad=int(bad.sum()), bad_idx=np.nonzero(bad)[0][:10].tolist(),
                n_excused_fail=int((over & excused).sum()),
                frac_excused_fail=float((over & excused).mean()) if rel.size else 0.0)


def assert_costs(S_gpu, S_orc, margin, max_excused_fail=0.0):
    """Every sample within S_REL_TOL, except (when max_excused_fail > 0) at most that share of
    the samples, each of them within MARGIN_EXCUSE of a cost jump."""
    assert max_excused_fail <= MAX_EXCUSED_FAIL
    r = cost_report(S_gpu, S_orc, margin)
    assert r["n_bad"] == 0, f"sample costs outside tolerance: {r}"
    assert r["frac_excused_fail"] <= max_excused_fail, f"samples near a cost jump outside tolerance: {r}"
    if max_excused_fail == 0.0:
        assert r["max_rel_all"] <= S_REL_TOL, r
    return r


def assert_update(u_gpu, x_gpu, orc):
    """u* and x* against the oracle's, whatever the argmin."""
    np.testing.assert_allclose(u_gpu, orc.u_star, rtol=0, atol=U_ABS_TOL)
    np.testing.assert_allclose(x_gpu, orc.x_star, rtol=0, atol=X_ABS_TOL)


def argmin_ok(argmin_gpu, S_orc):
    order = np.argsort(S_orc, kind="stable")
    s1 = S_orc[order[0]]
    near = np.nonzero(S_orc - s1 <= NEAR_TIE * max(abs(s1), 1.0))[0]
    if len(near) == 1:
        return argmin_gpu == order[0]
    return argmin_gpu in set(near.tolist())
