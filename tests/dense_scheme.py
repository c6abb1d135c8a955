"""Second, independent FP64 implementation of SSPRK2-SE / SSPRK3-SE for tiny
meshes, written with every horizontal operator assembled as a dense matrix.

Test infrastructure: it exists only to check the C oracle by brute force.  It
shares no code with the oracle or with the CUDA library; it reads the raw
mesh arrays (connectivity, lengths, areas, kite areas, TRiSK weights) and
builds

* Div   [C, E]  div_i F  = (1/A_i) sum_e n_{e,i} l_e F_e, from cellsOnEdge
  (the normal of edge e points out of c1 and into c2);
* Grad  [E, C]  grad_e phi = (phi_c2 - phi_c1) / d_e;
* Curl  [V, E]  curl_v u = (1/A_v) * counter-clockwise circulation of u over
  the dual triangle, from verticesOnEdge: the tangent t_e = k x n_e points from
  v1 to v2, so a dual edge is traversed along -n_e around v1 and +n_e around
  v2;
* Perp  [E, E]  u^perp_e = (1/d_e) sum_e' w_{e,e'} l_e' u_e' (Thuburn et al.);
* Kin   [C, E]  K_i = sum_e l_e d_e u_e^2 / (4 A_i);
* Avg   [E, C]  centred edge average;  Kite [V, C] kite-area average over the
  ocean cells of a vertex;  VAvg [E, V] mean of the edge's two vertices;
  Rot [E, V] (omega_v2 - omega_v1) / l_e.

The step follows the paper: the split (Eq. BBspl), Algorithm 1 (or
Algorithm 2 with a dense solve per edge column when vmix is set), the
barotropic SSPRK2/SSPRK3 sub-cycles of Algorithms 3 and 4 in Shu-Osher form,
the thickness and tracer stages with the z-star vertical velocity, and the
SSH reconciliation of Sec. 3.4 (modes off / printed / consistent).  Vertical
column operations are written with cumulative sums over whole [cells,
layers] arrays rather than loops.
"""
from __future__ import annotations

import numpy as np

RECON = {"off": 0, "paper": 1, "consistent": 2}


class DenseScheme:
    def __init__(self, m, L, p, rest_frac=None, max_level=None, rest_thickness=None):
        self.L = L
        self.p = dict(p)
        C, E, V = m.nCells, m.nEdges, m.nVertices
        c1, c2 = m.cellsOnEdge[:, 0], m.cellsOnEdge[:, 1]
        v1, v2 = m.verticesOnEdge[:, 0], m.verticesOnEdge[:, 1]
        ee = np.arange(E)
        l, d = m.dvEdge, m.dcEdge
        self.H = np.asarray(m.bottomDepth, float)
        # layers: a column keeps Kc layers, an edge the layers both its cells
        # keep; masks mc [C, L], me [E, L]; z-star shares s [C, L]
        self.Kc = np.full(C, L) if max_level is None else np.asarray(max_level)
        self.Ke = np.minimum(self.Kc[c1], self.Kc[c2])
        ks = np.arange(L)[None, :]
        self.mc = (ks < self.Kc[:, None]).astype(float)
        self.me = (ks < self.Ke[:, None]).astype(float)
        if rest_thickness is not None:
            self.s = np.asarray(rest_thickness, float) / self.H[:, None]
        else:
            frac = np.full(L, 1.0 / L) if rest_frac is None else np.asarray(rest_frac, float)
            self.s = np.tile(frac, (C, 1))

        Div = np.zeros((C, E))
        np.add.at(Div, (c1, ee), l / m.areaCell[c1])
        np.add.at(Div, (c2, ee), -l / m.areaCell[c2])
        Grad = np.zeros((E, C))
        np.add.at(Grad, (ee, c2), 1.0 / d)
        np.add.at(Grad, (ee, c1), -1.0 / d)
        Curl = np.zeros((V, E))
        np.add.at(Curl, (v2, ee), d / m.areaTriangle[v2])
        np.add.at(Curl, (v1, ee), -d / m.areaTriangle[v1])
        Rot = np.zeros((E, V))
        np.add.at(Rot, (ee, v2), 1.0 / l)
        np.add.at(Rot, (ee, v1), -1.0 / l)
        Perp = np.zeros((E, E))
        for e in range(E):
            for j in range(m.nEdgesOnEdge[e]):
                ep = m.edgesOnEdge[e, j]
                Perp[e, ep] += m.weightsOnEdge[e, j] * l[ep] / d[e]
        Kin = np.zeros((C, E))
        np.add.at(Kin, (c1, ee), 0.25 * l * d / m.areaCell[c1])
        np.add.at(Kin, (c2, ee), 0.25 * l * d / m.areaCell[c2])
        Avg = np.zeros((E, C))
        np.add.at(Avg, (ee, c1), 0.5)
        np.add.at(Avg, (ee, c2), 0.5)
        VAvg = np.zeros((E, V))
        np.add.at(VAvg, (ee, v1), 0.5)
        np.add.at(VAvg, (ee, v2), 0.5)
        Kite = np.zeros((V, C))
        for v in range(V):
            for j in range(3):
                c = m.cellsOnVertex[v, j]
                if c >= 0:
                    Kite[v, c] += m.kiteAreasOnVertex[v, j]
        fE = np.asarray(m.fEdge, float)
        self.fV = np.asarray(m.fVertex, float)
        self.Div, self.Grad, self.Curl, self.Rot = Div, Grad, Curl, Rot
        self.Perp, self.Kin, self.Avg, self.Kite, self.VAvg = Perp, Kin, Avg, Kite, VAvg
        # energy-neutral Coriolis operator: the weights times (f_e + f_e')/2
        self.Cor = Perp * 0.5 * (fE[:, None] + fE[None, :])
        self.Lap = Grad @ Div - Rot @ Curl
        ws = self.p.get("windStress")
        self.wind = np.zeros(E) if ws is None else np.asarray(ws, float)
        self.recon = RECON[self.p.get("recon", "consistent")]

    def he(self, h):
        """edge thickness, 0 where the edge has no layer"""
        return (self.Avg @ h) * self.me

    def hv(self, h):
        """kite average over the cells active in the layer, 0 where none is"""
        num, den = self.Kite @ (h * self.mc), self.Kite @ self.mc
        return np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)

    # ---------------------------------------------------------------- vertical
    def w_interfaces(self, h, v):
        """z-star w[C, L+1] from d h_k/dt = s_k d(sum h)/dt (interface k = top of k)."""
        dv = self.Div @ (self.he(h) * v)                    # div(h_e v)_k  [C, L]
        tot = dv.sum(axis=1, keepdims=True)
        src = -dv + self.s * tot                            # w_k - w_{k+1} (0 below)
        w = np.zeros((h.shape[0], self.L + 1))
        w[:, :self.L] = np.cumsum(src[:, ::-1], axis=1)[:, ::-1]
        w[:, 0] = 0.0
        return w

    def rho(self, tr):
        p = self.p
        r = p["eos_rho_ref"] - p["eos_alpha"] * (tr[0] - p["eos_T_ref"])
        if tr.shape[0] >= 2:
            r = r + p["eos_beta"] * (tr[1] - p["eos_S_ref"])
        return r

    # ------------------------------------------------------------- baroclinic
    def rhs(self, u, ut, zeta, h, tr, vvisc_on=True):
        p, L = self.p, self.L
        g, rho0 = p["g"], p["rho0"]
        he = self.he(h)
        omega = self.Curl @ u
        hv = self.hv(h)
        q = np.where(hv > 0, (omega + self.fV[:, None]) / np.where(hv > 0, hv, 1.0), 0.0)
        qe = self.VAvg @ q                                    # mean of the edge's two vertices
        Q = np.stack([(self.Perp * 0.5 * (qe[:, k][:, None] + qe[:, k][None, :])) @ (he[:, k] * u[:, k])
                      for k in range(L)], axis=1)
        Cu, Cut = self.Cor @ u, self.Cor @ ut
        K = self.Kin @ (u * u)
        rho = self.rho(tr)
        rh = rho * h
        pres = g * (np.cumsum(rh, axis=1) - 0.5 * rh)
        below = np.cumsum(h[:, ::-1], axis=1)[:, ::-1] - h   # sum_{l>k} h_l
        zmid = -self.H[:, None] + below + 0.5 * h
        pgf = (self.Grad @ pres + g * (self.Avg @ rho) * (self.Grad @ zmid)) / rho0
        w = self.w_interfaces(h, u)
        we = self.Avg @ w                                    # [E, L+1]
        E = u.shape[0]
        ee = np.arange(E)
        inner = (np.arange(L + 1)[None, :] >= 1) & (np.arange(L + 1)[None, :] < self.Ke[:, None])
        Dz = np.zeros((E, L + 1))                            # D_zt(u) at interior interfaces
        hi = 0.5 * (he[:, :-1] + he[:, 1:])
        Dz[:, 1:L] = (u[:, :-1] - u[:, 1:]) / np.where(hi > 0, hi, 1.0)
        Dz = np.where(inner, Dz, 0.0)
        wD = we * Dz
        vadv = 0.5 * (wD[:, :L] + wD[:, 1:])
        X = p["nu_v"] * Dz
        X[:, 0] = self.wind / rho0
        kb = self.Ke - 1                                     # the edge's bottom layer
        ubot = u[ee, kb]
        speed = np.sqrt(ubot ** 2 + (self.Perp @ u)[ee, kb] ** 2)
        X[ee, self.Ke] = p["c_drag"] * speed * ubot
        vvisc = (X[:, :L] - X[:, 1:]) / np.where(he > 0, he, 1.0) if vvisc_on else 0.0
        bih = self.Lap @ ((self.Lap @ u) * self.me)          # del^4 u (del^2 u on edge layers)
        return self.me * (Cut + (Q - Cu) - self.Grad @ K - pgf - vadv + p["nu_h"] * (self.Lap @ u) + vvisc
                + g * (self.Grad @ zeta)[:, None] - p.get("nu_4", 0.0) * bih)

    def alg1(self, u, ut, zeta, h, tr, dt):
        ut1 = ut + dt * self.rhs(u, ut, zeta, h, tr)
        he = self.he(h)
        G = (he * ut1).sum(1) / he.sum(1) / dt
        return (ut1 - dt * G[:, None]) * self.me, G

    def alg2(self, u, ut, ub, zeta, h, tr, dt):
        """Algorithm 2: explicit stage without D^u, G, then for every edge the
        dense linear system (I - dt D^u) u1 = ut1 + ubar solved directly, wind
        explicit, drag c_d |u| u1 with the speed of the input u."""
        p = self.p
        ut1 = ut + dt * self.rhs(u, ut, zeta, h, tr, vvisc_on=False)
        he = self.he(h)
        G = (he * ut1).sum(1) / he.sum(1) / dt
        ut1 = (ut1 - dt * G[:, None]) * self.me
        utan = self.Perp @ u
        out = np.zeros_like(ut1)
        for e in range(u.shape[0]):
            K = int(self.Ke[e])
            hk = he[e, :K]
            A = np.eye(K)
            for k in range(K):
                if k >= 1:
                    c = dt * p["nu_v"] / (hk[k] * 0.5 * (hk[k - 1] + hk[k]))
                    A[k, k] += c
                    A[k, k - 1] -= c
                if k + 1 <= K - 1:
                    c = dt * p["nu_v"] / (hk[k] * 0.5 * (hk[k] + hk[k + 1]))
                    A[k, k] += c
                    A[k, k + 1] -= c
            speed = np.hypot(u[e, K - 1], utan[e, K - 1])
            A[K - 1, K - 1] += dt * p["c_drag"] * speed / hk[K - 1]
            r = ut1[e, :K] + ub[e]
            r[0] += dt * self.wind[e] / p["rho0"] / hk[0]
            out[e, :K] = np.linalg.solve(A, r) - ub[e]
        return out, G

    def bcl(self, u, ut, ub, zeta, h, tr, dt):
        if self.p.get("vmix"):
            return self.alg2(u, ut, ub, zeta, h, tr, dt)
        return self.alg1(u, ut, zeta, h, tr, dt)

    # ------------------------------------------------------------- barotropic
    def btr_fe(self, ub, z, G, tau):
        flux = ub * (self.Avg @ (z + self.H))
        return (ub + tau * (self.Cor @ ub - self.p["g"] * (self.Grad @ z) + G),
                z - tau * (self.Div @ flux), flux)

    def subcycle(self, order, ub, z, G, dt, M):
        tau = dt / M
        F = np.zeros_like(ub)
        for _ in range(M):
            u1, z1, f0 = self.btr_fe(ub, z, G, tau)
            u2, z2, f1 = self.btr_fe(u1, z1, G, tau)
            if order == 2:
                ub, z = 0.5 * (ub + u2), 0.5 * (z + z2)
                F += (f0 + f1) / (2 * M)
            else:
                u3, z3, f2 = self.btr_fe(0.75 * ub + 0.25 * u2, 0.75 * z + 0.25 * z2, G, tau)
                ub, z = ub / 3 + 2 * u3 / 3, z / 3 + 2 * z3 / 3
                F += (f0 + f1) / (6 * M) + 2 * f2 / (3 * M)
        return ub, F, z

    # ------------------------------------------------------ thickness, tracers
    def thick(self, h, tr, v, dt):
        p, L = self.p, self.L
        he = self.he(h)
        F = he * v
        w = self.w_interfaces(h, v)
        h1 = h + dt * (-(self.Div @ F) - (w[:, :L] - w[:, 1:]))
        inner = (np.arange(L + 1)[None, :] >= 1) & (np.arange(L + 1)[None, :] < self.Kc[:, None])
        out = []
        for phi in tr:
            adv = self.Div @ (F * (self.Avg @ phi))
            dif = self.Div @ (he * p["kappa_h"] * (self.Grad @ phi))
            pt = np.zeros((h.shape[0], L + 1))
            pt[:, 1:L] = 0.5 * (phi[:, :-1] + phi[:, 1:])
            vf = np.where(inner, pt, 0.0) * w
            dz = np.zeros((h.shape[0], L + 1))
            hi = 0.5 * (h[:, :-1] + h[:, 1:])
            dz[:, 1:L] = (phi[:, :-1] - phi[:, 1:]) / np.where(hi > 0, hi, 1.0)
            dz = np.where(inner, dz, 0.0)
            hphi = h * phi + dt * (-adv - (vf[:, :L] - vf[:, 1:]) + dif
                                   + p["kappa_v"] * (dz[:, :L] - dz[:, 1:]))
            out.append(np.where(self.mc > 0, hphi / np.where(h1 > 0, h1, 1.0), 0.0))
        return h1, np.stack(out)

    # --------------------------------------------------------------- the step
    def split(self, u, h):
        he = self.he(h)
        ub = (he * u).sum(1) / he.sum(1)
        return ub, (u - ub[:, None]) * self.me

    def colflux(self, u, h):
        he = self.he(h)
        return (he * u).sum(1), he.sum(1)

    def full(self, ub, ut):
        """u = ubar + utilde where the edge has a layer, 0 elsewhere"""
        return (ub[:, None] + ut) * self.me

    def comb(self, a, h1, p1, b, h2, p2, hn):
        return np.where(self.mc > 0, (a * h1 * p1 + b * h2 * p2) / np.where(hn > 0, hn, 1.0), 0.0)

    def step(self, order, dt, M, u, h, tr):
        r = self.recon
        zn = h.sum(1) - self.H
        ubn, utn = self.split(u, h)
        ut1, G0 = self.bcl(u, utn, ubn, zn, h, tr, dt)
        ub1, Fz1, _ = self.subcycle(order, ubn, zn, G0, dt, M)
        u1 = self.full(ub1, ut1)
        Fh1, hsn = self.colflux(u, h)
        D1 = Fz1 - Fh1
        v = (u + (D1 / hsn)[:, None] * (r > 0)) * self.me
        h1, tr1 = self.thick(h, tr, v, dt)
        z1 = h1.sum(1) - self.H
        if order == 2:
            ut2, G1 = self.bcl(u1, ut1, ub1, z1, h1, tr1, dt)
            utn1 = 0.5 * (utn + ut2)
            ubn1, Fz2, _ = self.subcycle(2, ubn, zn, 0.5 * (G0 + G1), dt, M)
            un1 = self.full(ubn1, utn1)
            f2, hs1 = self.colflux(un1, h1)
            Fh2 = 0.5 * ((Fz1 if r == 2 else Fh1) + f2)
            D2 = Fz2 - Fh2
            v = (un1 + (2.0 * D2 / hs1)[:, None] * (r > 0)) * self.me
            h2, tr2 = self.thick(h1, tr1, v, dt)
            hn1 = 0.5 * (h + h2)
            trn1 = self.comb(0.5, h, tr, 0.5, h2, tr2, hn1)
            return un1, hn1, trn1
        ut2, G1 = self.bcl(u1, ut1, ub1, z1, h1, tr1, dt)
        uth = 0.75 * utn + 0.25 * ut2
        ub2, Fz2, _ = self.subcycle(3, ub1, z1, G1, dt, M)
        ubh = 0.75 * ubn + 0.25 * ub2
        uh = self.full(ubh, uth)
        Fh2, hs1 = self.colflux(u1, h1)
        D2 = Fz2 - Fh2
        v = (u1 + (D2 / hs1)[:, None] * (r > 0)) * self.me
        h2, tr2 = self.thick(h1, tr1, v, dt)
        hh = 0.75 * h + 0.25 * h2
        trh = self.comb(0.75, h, tr, 0.25, h2, tr2, hh)
        zh = hh.sum(1) - self.H
        ut3, G2 = self.bcl(uh, uth, ubh, zh, hh, trh, dt)
        utn1 = utn / 3 + 2 * ut3 / 3
        ubn1, Fz3, _ = self.subcycle(3, ubn, zn, G0 / 6 + G1 / 6 + 2 * G2 / 3, dt, M)
        un1 = self.full(ubn1, utn1)
        hen, he1, heh = self.he(h), self.he(h1), self.he(hh)
        if r == 2:
            Fh3 = (Fz1 + Fz2) / 6 + (2 * (u + un1) * heh).sum(1) / 6
        else:
            Fh3 = ((u * hen + u1 * he1 + 2 * (u + un1) * heh) / 6).sum(1)
        D3 = Fz3 - Fh3
        v = (0.5 * (u + un1) + (1.5 * D3 / heh.sum(1))[:, None] * (r > 0)) * self.me
        h3, tr3 = self.thick(hh, trh, v, dt)
        hn1 = h / 3 + 2 * h3 / 3
        trn1 = self.comb(1 / 3, h, tr, 2 / 3, h3, tr3, hn1)
        return un1, hn1, trn1
