"""The border, clamp and near-plane stress scene of the GPU parity tests
(test_conservative_cull_keeps_every_reaching_pair) reaches the cases it is
meant to, by the oracle's own visibility rule: pairs whose cutoff ellipse
reaches a pixel centre from a centre outside the image, with the Jacobian
clamp active, and at the near plane.  CPU only."""
import numpy as np

import oracle
from tests.test_parity_gpu import _edge_stress


def test_edge_stress_scene_reaches_its_cases():
    sc = _edge_stress()
    visible = outside = clamped = near = 0
    for c in sc.cameras:
        P = oracle.project(sc, camera=c)
        for g in np.nonzero(P["valid"])[0]:
            d2max = min(9.0, 2.0 * np.log(255.0 * P["opacity"][g]))
            if not d2max >= 0:
                continue
            q = oracle._quad_min_over_box(P["conic0"][g], P["conic1"][g], P["conic2"][g], P["u"][g], P["v"][g],
                                          0.0, c.W - 1.0, 0.0, c.H - 1.0)
            if q > d2max:
                continue
            visible += 1
            outside += not (0 <= P["u"][g] <= c.W - 1 and 0 <= P["v"][g] <= c.H - 1)
            clamped += bool(P["clamp_x"][g] or P["clamp_y"][g])
            near += P["z"][g] < 0.26
    assert visible > 1000, visible
    assert outside > 300 and clamped > 100 and near > 20, (outside, clamped, near)
    # the cameras sit far from the world origin: the camera transform cancels large terms
    assert np.abs(sc.means).max() > 1000.0
