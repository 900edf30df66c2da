"""Surface offsetting (Sec. 4): offset points from the GPU normals against the
oracle, and the same-parameterisation refit by fused Adam steps converging to
them (closer than the direct control-point offset, as the paper reports)."""
import numpy as np
import pytest

from gpu_util import S_TOL, bbox_diag
from oracle import oracle as O
from paper_2104_14547_gb300 import offset, synth

pytestmark = pytest.mark.gpu


def test_offset_targets_and_refit():
    d = 0.02
    surfs = synth.offset_batch(3, batch=5)
    fit = offset.OffsetFit(surfs, d)
    T = fit.target.cpu().numpy()
    a = 0
    for s in surfs:
        S, _, _, N = O.surface_derivs(s.p, s.q, s.U, s.V, s.ctrl, s.u, s.v)
        ref = (S + d * N).reshape(-1, 3)
        n = ref.shape[0]
        assert np.abs(T[a: a + n] - ref).max() <= S_TOL * bbox_diag(s.ctrl) + 2e-4 * d
        a += n
    before = fit.deviation()
    assert np.all(before <= d * (1 + 1e-4)) and np.all(before >= 0.9 * d)   # the base surface sits d away
    cp = fit.control_point_offset_deviation()
    fit.run(300, lr=2e-3)
    after = fit.deviation()
    assert np.all(after <= 0.05 * d), after / d
    assert np.all(after < cp), (after, cp)
    assert float(fit.loss.sum()) > 0.0
