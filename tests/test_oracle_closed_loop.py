"""The oracle's disturbed closed loop (Eq. 26, Alg. 2) against the paper's
qualitative result (Sec. VI): the shield lowers how often the executed
trajectory breaks the DCBF condition h(x_{n+1}) >= (1 - alpha) h(x_n)
(Eq. 17) and how often it ends outside the track (h < 0, Eq. 23).

Plain MPPI here is the controller without the shield and without the CBF term
in the cost (C = 0); Shield-MPPI adds the CBF cost (C = 1000) and ten Armijo
repair iterations of V+ before v_0 is executed.  Both run on the same narrow
tracks (half-width 1-1.5 m), target speed 14 m/s and disturbances (std 0.6 on
v_y and r, the same Philox stream), K = 64, T = 20, 40 updates per problem.
The counts themselves belong to this synthetic setup; only the ordering is
the paper's.
"""
import numpy as np

from paper_2302_11719_gb300 import inputs as I


def _closed_loop(orc, seed, shield, n_inst=8, n_up=40):
    ib = I.uneven_instances(n_inst=n_inst, seed=seed, K_lo=64, K_hi=64, T_lo=20, T_hi=20,
                            w_lo=1.0, w_hi=1.5, C_cbf=1000.0 if shield else 0.0, **I.HARSH)
    a = 1.0 - float(np.float32(ib.params[0]["alpha"]))
    viol = outside = 0
    for i in range(n_inst):
        m = orc.Model(ib.params[i], ib.tracks[i])
        x, V = ib.x0[i].astype(np.float64), np.zeros((20, 2))
        for n in range(n_up):
            x32, V32 = x.astype(np.float32), V.astype(np.float32)
            _, Vp = orc.mppi_step(m, x32, V32, n, i, nthreads=8)
            v = orc.repair(m, x32, Vp.astype(np.float32), 10)[0][0] if shield else Vp[0]
            x1 = orc.apply(m, x32, v, n, i)
            seg, d0 = orc.track_nearest(m, x32[3], x32[4])
            _, d1 = orc.track_follow(m, seg, x1[3], x1[4])
            h0, h1 = orc.h(m, d0), orc.h(m, d1)
            viol += h1 < a * h0
            outside += h1 < 0.0
            x, V = x1, orc.shift(m, Vp)
    return viol, outside


def test_shield_lowers_violations_in_closed_loop(orc):
    tot_p = tot_s = 0
    for seed in range(5):
        vp, op = _closed_loop(orc, seed, shield=False)
        vs, os_ = _closed_loop(orc, seed, shield=True)
        print("seed %d: DCBF-condition violations plain %d, shield %d; outside %d / %d"
              % (seed, vp, vs, op, os_))
        assert vs <= vp and os_ <= op
        tot_p += vp
        tot_s += vs
    assert tot_s < tot_p
