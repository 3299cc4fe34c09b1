"""The FP64 oracle driven through coupled levels in the schedule of the library's level hierarchy
(test infrastructure: orchestration of oracle.Sim and oracle.Coupler, no method arithmetic of
its own beyond the leapfrog bookkeeping stated below).

Schedule of one coupling period T: every level advances T / dt_l steps with its held external
forces; then the held forces are cleared and the couplers run finest pair last, each adding its
forces.  A coupler acts on the leapfrog state the GPU keeps: positions at the integer step,
velocities at the half step before it (v - dt/2 F/m, w - dt/2 T/I), contact forces with the
stored overlaps of that step.  Held forces act from the step at which they are set (the forces
of that step are updated by the change).  Inserted particles join with the coupler's velocity
as their half-step velocity, no spin, no force at the step of insertion, IDs handed out in
insertion order; removed particles leave at once (their IDs are not reused).
"""
import numpy as np

import oracle


class OracleLevels:
    def __init__(self, P, wls, specs, band_q=4.0):
        self.P = P
        self.dt = [float(p[5]) for p in P]
        T = specs[0]["interval"] * self.dt[1]
        self.steps = [int(round(T / dt)) for dt in self.dt]
        self.sims = [oracle.Sim(p, wl.x, wl.v, wl.w, wl.r, wl.m) for p, wl in zip(P, wls)]
        self.next_id = [wl.n for wl in wls]
        self.fext = [np.zeros((wl.n, 3)) for wl in wls]
        self.cps = []
        for k, sp in enumerate(specs):
            fine = wls[k + 1]
            qf = oracle.quantum(fine.lo, fine.hi)
            cp = oracle.Coupler(sp, P[k], P[k + 1], float(np.max(fine.r)), fine.material.rho,
                                idcap=int(1.5 * wls[k].n) + 100_000, band=band_q * qf)
            cp.record(wls[k].x, np.arange(wls[k].n))
            self.cps.append(cp)
        self.outs = []

    def _state(self, k):
        s = self.sims[k]
        dt = self.dt[k]
        I = 0.4 * s.m * s.r ** 2
        ha, hb, hx, _ = s.history()
        return dict(x=s.x, v=s.v - 0.5 * dt * s.F / s.m[:, None], w=s.w - 0.5 * dt * s.T / I[:, None], r=s.r,
                    m=s.m, id=s.id, hist=(ha, hb, hx))

    def _replace(self, k, x, v, w, r, m, ids, F, T, hist, fext):
        old = self.sims[k]
        s = oracle.Sim(old.P, x, v, w, r, m, ids=ids)
        ha, hb, hx, sl = hist
        keep = np.isin(ha, ids) & ((hb < 0) | np.isin(hb, ids))
        n = int(keep.sum())
        s.ha[:n], s.hb[:n], s.hxi[:n], s.slip[:n] = ha[keep], hb[keep], hx[keep], sl[keep]
        s.nh[0] = n
        s.F[:] = F
        s.T[:] = T
        s.primed = old.primed
        self.sims[k] = s
        self.fext[k] = fext

    def advance(self, periods=1):
        for _ in range(periods):
            for k, s in enumerate(self.sims):
                s.fext = self.fext[k]
                s.run(self.steps[k])
            new = [np.zeros_like(f) for f in self.fext]
            outs = []
            for k, cp in enumerate(self.cps):
                out = cp.call(self._state(k), self._state(k + 1), 0.0, 0.0)
                outs.append(out)
                new[k] += out["fext_c"]
                new[k + 1] += out["fext_f"]
                # removal, then insertion, on the fine side
                s = self.sims[k + 1]
                live = out["removed"] == 0
                ins = [(c, t) for c in range(len(out["nins"])) for t in range(out["nins"][c])]
                ni = len(ins)
                xi = np.array([out["ins_x"][c, t, :3] for c, t in ins]).reshape(ni, 3)
                ri = np.array([out["ins_x"][c, t, 3] for c, t in ins])
                mi = np.array([out["ins_m"][c, t] for c, t in ins])
                fav = out["fav"]
                vi = np.array([fav[c, 1:4] / fav[c, 0] if fav[c, 0] > 0 else np.zeros(3) for c, _ in ins]).reshape(ni, 3)
                ids = np.concatenate([s.id[live], self.next_id[k + 1] + np.arange(ni)])
                self.next_id[k + 1] += ni
                self._replace(k + 1, np.vstack([s.x[live], xi]), np.vstack([s.v[live], vi]),
                              np.vstack([s.w[live], np.zeros((ni, 3))]), np.concatenate([s.r[live], ri]),
                              np.concatenate([s.m[live], mi]), ids, np.vstack([s.F[live], np.zeros((ni, 3))]),
                              np.vstack([s.T[live], np.zeros((ni, 3))]), s.history(),
                              np.vstack([self.fext[k + 1][live], np.zeros((ni, 3))]))
                new[k + 1] = np.vstack([new[k + 1][live], np.zeros((ni, 3))])
            # the new held forces act from this step: F and the integer-step velocity follow
            for k, s in enumerate(self.sims):
                dF = new[k] - self.fext[k]
                s.F = s.F + dF
                s.v = s.v + 0.5 * self.dt[k] * dF / s.m[:, None]
                self.fext[k] = new[k]
            self.outs.append(outs)
        return self

    def positions_by_id(self, k, nid):
        """(nid, 3) positions indexed by particle ID, NaN where removed."""
        out = np.full((nid, 3), np.nan)
        s = self.sims[k]
        out[s.id] = s.x
        return out
