"""Comparison rules between the CUDA path and the FP64 oracle.

Tolerances (the planner's accuracy targets):
* per-sample cost S: |S_gpu - S_oracle| <= 1e-4 * max(|S_oracle|, 1);
* updated controls u* and the optimal trajectory x*: 1e-4 absolute;
* Philox words: bit-exact; argmin index: exact unless the oracle's two lowest
  costs are within 1e-4 relative (a near tie), where the GPU's index must lie in
  the oracle's near-tie set.

The step cost has jumps (the reference yaw switches between polyline segments,
c_target's indicator, the collision-only switch, the yaw wrap).  The oracle
reports, per sample, how far (metres / radians) the rollout passed from the
nearest jump; a sample whose margin is below MARGIN_EXCUSE may land on the other
side in binary32 and is excused from the cost tolerance (and counted).
"""
import numpy as np

S_REL_TOL = 1e-4
U_ABS_TOL = 1e-4
X_ABS_TOL = 1e-4
MARGIN_EXCUSE = 1e-5
NEAR_TIE = 1e-4


def cost_report(S_gpu, S_orc, margin):
    rel = np.abs(S_gpu - S_orc) / np.maximum(np.abs(S_orc), 1.0)
    excused = margin < MARGIN_EXCUSE
    bad = (rel > S_REL_TOL) & ~excused
    return dict(max_rel=float(rel[~excused].max()) if (~excused).any() else 0.0,
                max_rel_all=float(rel.max()), excused=int(excused.sum()), frac_excused=float(excused.mean()),
                n_bad=int(bad.sum()), bad_idx=np.nonzero(bad)[0][:10].tolist())


def assert_costs(S_gpu, S_orc, margin, max_excused_frac=0.02):
    r = cost_report(S_gpu, S_orc, margin)
    assert r["n_bad"] == 0, f"sample costs outside tolerance: {r}"
    assert r["frac_excused"] <= max_excused_frac, f"too many samples near a cost jump: {r}"
    return r


def argmin_ok(argmin_gpu, S_orc):
    order = np.argsort(S_orc, kind="stable")
    s1 = S_orc[order[0]]
    near = np.nonzero(S_orc - s1 <= NEAR_TIE * max(abs(s1), 1.0))[0]
    if len(near) == 1:
        return argmin_gpu == order[0]
    return argmin_gpu in set(near.tolist())
