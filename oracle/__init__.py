"""ctypes wrapper of the FP64 CPU oracle (oracle/sse_oracle.c).

TEST INFRASTRUCTURE ONLY.  Imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; the product path never imports
it.  It shares no code with the CUDA library.

All arrays are numpy float64, layer-fastest: u[E, L], h[C, L], tracers
[nT, C, L].  ``mesh`` is any object with the attributes of
``paper_2105_13484_gb300.mesh.Mesh`` (duck-typed; nothing is imported from the
product package).
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sse_oracle.c")
_LIB = os.path.join(_HERE, "libsse_oracle.so")
_LIB_OMP = os.path.join(_HERE, "libsse_oracle_omp.so")
_SRC_COUNT = os.path.join(_HERE, "flop_count.cpp")
_LIB_COUNT = os.path.join(_HERE, "libsse_oracle_count.so")

_dp = ct.POINTER(ct.c_double)
_ip = ct.POINTER(ct.c_int)


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, no FMA contraction).  With
    ``openmp`` a second library is built from the same source with -fopenmp:
    its loops over cells, edges and vertices run across threads and give
    results bit-identical to the serial library (each iteration writes only
    its own entity's outputs)."""
    lib = _LIB_OMP if openmp else _LIB
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "sse_oracle.h"))):
        tmp = lib + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-shared", "-fPIC",
                               *(["-fopenmp"] if openmp else []), _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, lib)
    return lib


def build_counting(force: bool = False) -> str:
    """Compile the counting build (flop_count.cpp: the oracle's source with
    every double an operation-counting wrapper), serial, no FMA contraction."""
    deps = [_SRC, _SRC_COUNT, os.path.join(_HERE, "sse_oracle.h")]
    if force or not os.path.exists(_LIB_COUNT) or os.path.getmtime(_LIB_COUNT) < max(
            os.path.getmtime(d) for d in deps):
        tmp = _LIB_COUNT + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared",
                               "-fPIC", "-I", _HERE, _SRC_COUNT, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_COUNT)
    return _LIB_COUNT


def host_threads() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class _Mesh(ct.Structure):
    _fields_ = [("nCells", ct.c_int), ("nEdges", ct.c_int), ("nVertices", ct.c_int),
                ("maxEdges", ct.c_int), ("maxEdges2", ct.c_int), ("nLayers", ct.c_int),
                ("cellsOnEdge", _ip), ("verticesOnEdge", _ip), ("nEdgesOnCell", _ip),
                ("edgesOnCell", _ip), ("cellsOnVertex", _ip), ("edgesOnVertex", _ip),
                ("nEdgesOnEdge", _ip), ("edgesOnEdge", _ip), ("weightsOnEdge", _dp),
                ("dcEdge", _dp), ("dvEdge", _dp), ("areaCell", _dp), ("areaTriangle", _dp),
                ("kiteAreasOnVertex", _dp), ("fEdge", _dp), ("fVertex", _dp),
                ("bottomDepth", _dp), ("restThicknessFrac", _dp), ("maxLevelCell", _ip),
                ("restThickness", _dp)]


class _Params(ct.Structure):
    _fields_ = [("nTracers", ct.c_int), ("recon", ct.c_int)] + [
        (n, ct.c_double) for n in ("g", "rho0", "nu_h", "nu_v", "kappa_h", "kappa_v", "c_drag",
                                   "eos_rho_ref", "eos_alpha", "eos_beta", "eos_T_ref",
                                   "eos_S_ref")] + [("windStress", _dp), ("vmix", ct.c_int),
                                                     ("nu_4", ct.c_double)]


class _Aux(ct.Structure):
    _fields_ = [(n, _dp) for n in ("zeta_sub", "D1", "D2", "D3", "Fz1", "Fz2", "Fz3", "G0",
                                   "G1", "G2")]


RECON = {"off": 0, "paper": 1, "consistent": 2}

DEFAULT_PARAMS = dict(nTracers=1, recon="consistent", g=9.80616, rho0=1000.0, nu_h=0.0, nu_v=0.0,
                      kappa_h=0.0, kappa_v=0.0, c_drag=0.0, eos_rho_ref=1000.0, eos_alpha=0.2,
                      eos_beta=0.8, eos_T_ref=10.0, eos_S_ref=35.0, windStress=None, vmix=0, nu_4=0.0)


def _d(a):
    return a.ctypes.data_as(_dp)


class Oracle:
    """FP64 oracle bound to one mesh, layer count and parameter set."""

    def __init__(self, mesh, nLayers: int, params: dict | None = None, rest_frac=None,
                 max_level=None, rest_thickness=None, threads: int = 1, counting: bool = False):
        """max_level [C] / rest_thickness [C, L]: partial bottom cells (both or
        neither; without them every column has all layers).  threads > 1 runs
        the OpenMP build of the same source on that many host threads;
        counting runs the operation-counting build (serial; see flops())."""
        self.threads = 1 if counting else max(1, int(threads))
        self.counting = bool(counting)
        self.lib = ct.CDLL(build_counting() if counting else build(openmp=self.threads > 1))
        self._sig()
        if counting:
            self.lib.om_flops_read.restype = ct.c_ulonglong
            self.lib.om_flops_reset()
        if self.threads > 1:
            self.lib.om_set_threads(self.threads)
        self.L = int(nLayers)
        self.C, self.E, self.V = int(mesh.nCells), int(mesh.nEdges), int(mesh.nVertices)
        self._keep = []

        def ia(x):
            a = np.ascontiguousarray(x, dtype=np.int32)
            self._keep.append(a)
            return a.ctypes.data_as(_ip)

        def da(x):
            a = np.ascontiguousarray(x, dtype=np.float64)
            self._keep.append(a)
            return a.ctypes.data_as(_dp)

        if rest_frac is None:
            rest_frac = np.full(self.L, 1.0 / self.L)
        self.rest_frac = np.asarray(rest_frac, dtype=np.float64)
        self.bottomDepth = np.asarray(mesh.bottomDepth, dtype=np.float64)
        self.m = _Mesh(self.C, self.E, self.V, int(mesh.maxEdges), int(mesh.maxEdges2), self.L,
                       ia(mesh.cellsOnEdge), ia(mesh.verticesOnEdge), ia(mesh.nEdgesOnCell),
                       ia(mesh.edgesOnCell), ia(mesh.cellsOnVertex), ia(mesh.edgesOnVertex),
                       ia(mesh.nEdgesOnEdge), ia(mesh.edgesOnEdge), da(mesh.weightsOnEdge),
                       da(mesh.dcEdge), da(mesh.dvEdge), da(mesh.areaCell), da(mesh.areaTriangle),
                       da(mesh.kiteAreasOnVertex), da(mesh.fEdge), da(mesh.fVertex),
                       da(mesh.bottomDepth), da(self.rest_frac),
                       None if max_level is None else ia(max_level),
                       None if rest_thickness is None else da(rest_thickness))
        self.set_params(params or {})

    def set_params(self, params: dict):
        q = dict(DEFAULT_PARAMS)
        q.update(params)
        self.params = q
        recon = q["recon"]
        recon = RECON[recon] if isinstance(recon, str) else int(recon)
        self.nT = int(q["nTracers"])
        ws = q.get("windStress")
        if ws is not None:
            self._ws = np.ascontiguousarray(ws, dtype=np.float64)
            wsp = _d(self._ws)
        else:
            self._ws = None
            wsp = None
        self.p = _Params(self.nT, recon, *[float(q[n]) for n in (
            "g", "rho0", "nu_h", "nu_v", "kappa_h", "kappa_v", "c_drag", "eos_rho_ref",
            "eos_alpha", "eos_beta", "eos_T_ref", "eos_S_ref")], wsp, int(bool(q.get("vmix", 0))),
            float(q.get("nu_4", 0.0)))

    def _sig(self):
        L = self.lib
        for n in ("om_div", "om_grad", "om_curl", "om_tangential", "om_kinetic_energy",
                  "om_laplacian", "om_biharmonic", "om_coriolis", "om_edge_thickness",
                  "om_vertex_thickness"):
            getattr(L, n).argtypes = [ct.c_void_p, ct.c_int, _dp, _dp]
        L.om_pv_flux.argtypes = [ct.c_void_p, ct.c_int, _dp, _dp, _dp]
        L.om_sse_step.restype = ct.c_int
        L.om_set_threads.argtypes = [ct.c_int]

    def flops(self, reset: bool = False) -> int:
        """FP64 operations (+, -, *, /, sqrt) the counting build has executed
        since the last reset in this process (one counter per library)."""
        if not self.counting:
            raise RuntimeError("flops() needs Oracle(..., counting=True)")
        n = int(self.lib.om_flops_read())
        if reset:
            self.lib.om_flops_reset()
        return n

    # ---- helpers -------------------------------------------------------
    @staticmethod
    def _f(x, shape=None):
        a = np.ascontiguousarray(x, dtype=np.float64)
        if shape is not None:
            a = a.reshape(shape)
        return a

    def _op(self, name, x, n_out, L=None):
        x = self._f(x)
        L = self.L if L is None else L
        out = np.zeros((n_out, L))
        getattr(self.lib, name)(ct.byref(self.m), L, _d(x), _d(out))
        return out

    # ---- TRiSK operators (x has shape [n, L] or [n]) ---------------------
    def _wrap(self, name, x, n_out):
        x = np.asarray(x, dtype=np.float64)
        flat = x.ndim == 1
        x2 = x.reshape(x.shape[0], -1)
        out = self._op(name, x2, n_out, L=x2.shape[1])
        return out[:, 0] if flat else out

    def div(self, F):
        return self._wrap("om_div", F, self.C)

    def grad(self, phi):
        return self._wrap("om_grad", phi, self.E)

    def curl(self, u):
        return self._wrap("om_curl", u, self.V)

    def tangential(self, u):
        return self._wrap("om_tangential", u, self.E)

    def kinetic_energy(self, u):
        return self._wrap("om_kinetic_energy", u, self.C)

    def laplacian(self, u):
        return self._wrap("om_laplacian", u, self.E)

    def biharmonic(self, u):
        return self._wrap("om_biharmonic", u, self.E)

    def coriolis(self, x):
        return self._wrap("om_coriolis", x, self.E)

    def edge_thickness(self, h):
        return self._wrap("om_edge_thickness", h, self.E)

    def vertex_thickness(self, h):
        return self._wrap("om_vertex_thickness", h, self.V)

    def pv_flux(self, u, h):
        u = np.asarray(u, dtype=np.float64)
        flat = u.ndim == 1
        u2 = self._f(u.reshape(u.shape[0], -1))
        h2 = self._f(np.asarray(h, dtype=np.float64).reshape(self.C, -1))
        Lx = u2.shape[1]
        out = np.zeros((self.E, Lx))
        self.lib.om_pv_flux(ct.byref(self.m), Lx, _d(u2), _d(h2), _d(out))
        return out[:, 0] if flat else out

    # ---- vertical pieces -----------------------------------------------
    def vertical_velocity(self, h, v):
        h, v = self._f(h), self._f(v)
        w = np.zeros((self.C, self.L + 1))
        self.lib.om_vertical_velocity(ct.byref(self.m), _d(h), _d(v), _d(w))
        return w

    def density(self, tr):
        tr = self._f(tr)
        rho = np.zeros((self.C, self.L))
        self.lib.om_density(ct.byref(self.m), ct.byref(self.p), _d(tr), _d(rho))
        return rho

    def pressure(self, h, rho):
        h, rho = self._f(h), self._f(rho)
        p = np.zeros((self.C, self.L))
        z = np.zeros((self.C, self.L))
        self.lib.om_pressure(ct.byref(self.m), ct.byref(self.p), _d(h), _d(rho), _d(p), _d(z))
        return p, z

    def ssh(self, h):
        h = self._f(h)
        z = np.zeros(self.C)
        self.lib.om_ssh(ct.byref(self.m), _d(h), _d(z))
        return z

    # ---- the split system ----------------------------------------------
    def split(self, u, h):
        u, h = self._f(u), self._f(h)
        ubar = np.zeros(self.E)
        ut = np.zeros((self.E, self.L))
        self.lib.om_split(ct.byref(self.m), _d(u), _d(h), _d(ubar), _d(ut))
        return ubar, ut

    def baroclinic_rhs(self, u, ut, zeta, h, tr):
        u, ut, zeta, h, tr = map(self._f, (u, ut, zeta, h, tr))
        out = np.zeros((self.E, self.L))
        self.lib.om_baroclinic_rhs(ct.byref(self.m), ct.byref(self.p), _d(u), _d(ut), _d(zeta),
                                   _d(h), _d(tr), _d(out))
        return out

    def baroclinic_feuler(self, u, ut, zeta, h, tr, dt):
        """Algorithm 1: returns (ut1 [E, L], G [E])."""
        u, ut, zeta, h, tr = map(self._f, (u, ut, zeta, h, tr))
        ut1 = np.zeros((self.E, self.L))
        G = np.zeros(self.E)
        self.lib.om_baroclinic_feuler(ct.byref(self.m), ct.byref(self.p), _d(u), _d(ut),
                                      _d(zeta), _d(h), _d(tr), ct.c_double(dt), _d(ut1), _d(G))
        return ut1, G

    def vertical_mixing_solve(self, u_drag, h, r, dt):
        """(I - dt D^u) x = r per edge column (the solve of Algorithm 2)."""
        u_drag, h, r = map(self._f, (u_drag, h, r))
        x = np.zeros((self.E, self.L))
        self.lib.om_vertical_mixing_solve(ct.byref(self.m), ct.byref(self.p), _d(u_drag), _d(h),
                                          _d(r), ct.c_double(dt), _d(x))
        return x

    def baroclinic_feuler_mixing(self, u, ut, ubar, zeta, h, tr, dt):
        """Algorithm 2: returns (ut1 [E, L], G [E])."""
        u, ut, ubar, zeta, h, tr = map(self._f, (u, ut, ubar, zeta, h, tr))
        ut1 = np.zeros((self.E, self.L))
        G = np.zeros(self.E)
        self.lib.om_baroclinic_feuler_mixing(ct.byref(self.m), ct.byref(self.p), _d(u), _d(ut),
                                             _d(ubar), _d(zeta), _d(h), _d(tr), ct.c_double(dt),
                                             _d(ut1), _d(G))
        return ut1, G

    def barotropic_fe(self, ubar, zeta, G, tau):
        ubar, zeta, G = map(self._f, (ubar, zeta, G))
        u1, z1, F = np.zeros(self.E), np.zeros(self.C), np.zeros(self.E)
        self.lib.om_barotropic_fe(ct.byref(self.m), ct.byref(self.p), _d(ubar), _d(zeta), _d(G),
                                  ct.c_double(tau), _d(u1), _d(z1), _d(F))
        return u1, z1, F

    def barotropic_substep(self, order, ubar, zeta, G, dt, M):
        """Algorithm 3 (order 2) / 4 (order 3): returns (ubar1, Fzeta, zeta1)."""
        ubar, zeta, G = map(self._f, (ubar, zeta, G))
        u1, Fz, z1 = np.zeros(self.E), np.zeros(self.E), np.zeros(self.C)
        self.lib.om_barotropic_substep(ct.byref(self.m), ct.byref(self.p), int(order), _d(ubar),
                                       _d(zeta), _d(G), ct.c_double(dt), int(M), _d(u1), _d(Fz),
                                       _d(z1))
        return u1, Fz, z1

    def thickness_tracer_fe(self, h, tr, v, dt):
        h, tr, v = map(self._f, (h, tr, v))
        h1 = np.zeros_like(h)
        tr1 = np.zeros_like(tr)
        self.lib.om_thickness_tracer_fe(ct.byref(self.m), ct.byref(self.p), _d(h), _d(tr), _d(v),
                                        ct.c_double(dt), _d(h1), _d(tr1))
        return h1, tr1

    def step(self, order, dt, M, u, h, tr, n_steps=1, aux=False):
        """n_steps SSPRK{order}-SE steps (copies; inputs untouched)."""
        u = self._f(u).copy()
        h = self._f(h).copy()
        tr = self._f(tr).reshape(self.nT, self.C, self.L).copy()
        rec = None
        for _ in range(n_steps):
            a = None
            if aux:
                rec = {"zeta_sub": np.zeros(self.C)}
                for n in ("D1", "D2", "D3", "Fz1", "Fz2", "Fz3", "G0", "G1", "G2"):
                    rec[n] = np.zeros(self.E)
                a = _Aux(*[_d(rec[n]) for n in ("zeta_sub", "D1", "D2", "D3", "Fz1", "Fz2",
                                                "Fz3", "G0", "G1", "G2")])
            rc = self.lib.om_sse_step(ct.byref(self.m), ct.byref(self.p), int(order),
                                      ct.c_double(dt), int(M), _d(u), _d(h), _d(tr),
                                      ct.byref(a) if a is not None else None)
            if rc != 0:
                raise ValueError(f"om_sse_step rejected its arguments (rc={rc})")
        return (u, h, tr, rec) if aux else (u, h, tr)
