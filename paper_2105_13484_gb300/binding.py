"""Thin ctypes binding of libsse.so (include/sse.h).

Argument marshalling only: every step of the method runs in the CUDA library.
Importing this module loads ``_lib/libsse.so`` and fails loudly if it is
missing; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsse.so")

SSE_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "BAD_MESH", -3: "OOM", -4: "CUDA", -5: "NONFINITE",
          -6: "SYNC_TIMEOUT", -7: "UNSUPPORTED"}
FP64, MIXED = 0, 1
OPT_VMIX = 1          # SSE_OPT_VMIX: Algorithm 2 (implicit vertical mixing)
RECON = {"off": 0, "paper": 1, "consistent": 2}
FIELD = {"u": 0, "h": 1, "tracer0": 2, "tracer1": 3, "wind": 4, "zeta": 5, "ubar": 6,
         "utilde": 7, "G": 8, "Fzeta": 9, "zeta_sub": 10}

_ip = ct.POINTER(ct.c_int32)
_dp = ct.POINTER(ct.c_double)


class SSEError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({code})")


class MeshDesc(ct.Structure):
    _fields_ = [("nCells", ct.c_int32), ("nEdges", ct.c_int32), ("nVertices", ct.c_int32),
                ("maxEdges", ct.c_int32), ("maxEdges2", ct.c_int32), ("nLayers", ct.c_int32),
                ("cellsOnEdge", _ip), ("verticesOnEdge", _ip), ("nEdgesOnCell", _ip),
                ("edgesOnCell", _ip), ("cellsOnVertex", _ip), ("edgesOnVertex", _ip),
                ("nEdgesOnEdge", _ip), ("edgesOnEdge", _ip), ("weightsOnEdge", _dp),
                ("dcEdge", _dp), ("dvEdge", _dp), ("areaCell", _dp), ("areaTriangle", _dp),
                ("kiteAreasOnVertex", _dp), ("fEdge", _dp), ("fVertex", _dp),
                ("bottomDepth", _dp), ("restThicknessFrac", _dp), ("maxLevelCell", _ip),
                ("restThickness", _dp)]


class Params(ct.Structure):
    _fields_ = [("precision", ct.c_int32), ("recon", ct.c_int32), ("nTracers", ct.c_int32),
                ("options", ct.c_int32)] + [
        (n, ct.c_double) for n in ("g", "rho0", "nu_h", "nu_v", "kappa_h", "kappa_v", "c_drag",
                                   "eos_rho_ref", "eos_alpha", "eos_beta", "eos_T_ref",
                                   "eos_S_ref", "nu_4")]


class Tuning(ct.Structure):
    _fields_ = [("patch_cells", ct.c_int32), ("bcl_patch_cells", ct.c_int32),
                ("reserved", ct.c_int32 * 6)]


TUNE = {"latency": 0, "throughput": 1}


class RequestInfo(ct.Structure):
    _fields_ = [("id", ct.c_int64), ("status", ct.c_int32), ("steps_done", ct.c_int32),
                ("t_submit", ct.c_double), ("t_admit", ct.c_double), ("t_done", ct.c_double),
                ("footprint", ct.c_size_t)]


class ServerInfo(ct.Structure):
    _fields_ = [("pending", ct.c_int32), ("active", ct.c_int32),
                ("max_active_seen", ct.c_int32), ("reserved", ct.c_int32),
                ("used_bytes", ct.c_size_t), ("peak_bytes", ct.c_size_t),
                ("budget_bytes", ct.c_size_t)]


class Diag(ct.Structure):
    _fields_ = [("volume", ct.c_double), ("tracer_content", ct.c_double * 2),
                ("kinetic_energy", ct.c_double), ("max_speed", ct.c_double),
                ("min_thickness", ct.c_double), ("zeta_min", ct.c_double),
                ("zeta_max", ct.c_double), ("step", ct.c_int64), ("nonfinite", ct.c_int32),
                ("reserved", ct.c_int32)]


EXPORTS = ["sse_mesh_create", "sse_mesh_destroy", "sse_state_create", "sse_state_destroy",
           "sse_state_init", "sse_probe_fma_rate", "sse_step_batch", "sse_server_create_ex",
           "sse_state_set", "sse_state_get", "sse_step", "sse_baroclinic_feuler",
           "sse_barotropic_substep", "sse_diagnostics", "sse_kernels_per_step", "sse_profile",
           "sse_profile_read", "sse_barotropic_substep_noalloc", "sse_state_footprint",
           "sse_state_footprint_ex", "sse_state_create_ex", "sse_state_patches", "sse_state_subcycle_shape",
           "sse_state_inject",
           "sse_state_set_f32", "sse_state_get_f32", "sse_state_graphs", "sse_state_transfer",
           "sse_state_sync",
           "sse_tune",
           "sse_mesh_dims", "sse_server_create", "sse_server_submit", "sse_server_query",
           "sse_server_wait", "sse_server_stats", "sse_server_release", "sse_server_destroy",
           "sse_strerror"]
KERNEL_CLASSES = ["cell_diag", "vertex", "edge_pre", "bcl_edge", "btr", "transport", "thickness",
                  "combine", "del4"]

_lib = None


def load(path: str = LIB_PATH):
    """Load libsse.so once; raise if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2105_13484_gb300.build.build()")
    lib = ct.CDLL(path)
    lib.sse_mesh_create.argtypes = [ct.POINTER(MeshDesc), ct.POINTER(ct.c_void_p)]
    lib.sse_mesh_destroy.argtypes = [ct.c_void_p]
    lib.sse_mesh_destroy.restype = None
    lib.sse_state_create.argtypes = [ct.c_void_p, ct.POINTER(Params), ct.c_void_p,
                                     ct.POINTER(ct.c_void_p)]
    lib.sse_state_destroy.argtypes = [ct.c_void_p]
    lib.sse_state_destroy.restype = None
    lib.sse_probe_fma_rate.argtypes = [ct.c_int, ct.POINTER(ct.c_double)]
    lib.sse_step_batch.argtypes = [ct.POINTER(ct.c_void_p), ct.c_int, ct.c_int,
                                   ct.POINTER(ct.c_double), ct.POINTER(ct.c_int32), ct.c_int,
                                   ct.c_void_p]
    lib.sse_state_init.argtypes = [ct.c_void_p, ct.POINTER(Params), ct.c_void_p, ct.c_void_p,
                                   ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                   ct.POINTER(ct.c_void_p)]
    lib.sse_state_set.argtypes = [ct.c_void_p, ct.c_int, ct.c_void_p]
    lib.sse_state_get.argtypes = [ct.c_void_p, ct.c_int, ct.c_void_p]
    lib.sse_step.argtypes = [ct.c_void_p, ct.c_int, ct.c_double, ct.c_int, ct.c_int]
    lib.sse_baroclinic_feuler.argtypes = [ct.c_void_p, ct.c_double]
    lib.sse_barotropic_substep.argtypes = [ct.c_void_p, ct.c_int, ct.c_double, ct.c_int]
    lib.sse_diagnostics.argtypes = [ct.c_void_p, ct.POINTER(Diag)]
    lib.sse_kernels_per_step.argtypes = [ct.c_void_p, ct.c_int]
    lib.sse_profile.argtypes = [ct.c_void_p, ct.c_int]
    lib.sse_profile_read.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_void_p]
    lib.sse_barotropic_substep_noalloc.argtypes = [
        ct.c_void_p, ct.c_int, ct.c_double, ct.c_int, ct.c_double, ct.c_void_p, ct.c_void_p,
        ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]
    lib.sse_state_footprint.argtypes = [ct.c_void_p, ct.POINTER(Params), ct.POINTER(ct.c_size_t)]
    lib.sse_mesh_dims.argtypes = [ct.c_void_p, ct.POINTER(ct.c_int32)]
    lib.sse_server_create.argtypes = [ct.c_int, ct.c_size_t, ct.c_int, ct.c_int, ct.c_int,
                                      ct.POINTER(ct.c_void_p)]
    lib.sse_server_create_ex.argtypes = [ct.c_int, ct.c_size_t, ct.c_int, ct.c_int, ct.c_int,
                                         ct.c_int, ct.POINTER(ct.c_void_p)]
    lib.sse_state_create_ex.argtypes = [ct.c_void_p, ct.POINTER(Params), ct.POINTER(Tuning),
                                        ct.c_void_p, ct.POINTER(ct.c_void_p)]
    lib.sse_state_footprint_ex.argtypes = [ct.c_void_p, ct.POINTER(Params), ct.POINTER(Tuning),
                                           ct.POINTER(ct.c_size_t)]
    lib.sse_state_patches.argtypes = [ct.c_void_p, ct.POINTER(ct.c_int)]
    lib.sse_state_subcycle_shape.argtypes = [ct.c_void_p, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]
    lib.sse_state_graphs.argtypes = [ct.c_void_p, ct.POINTER(ct.c_int)]
    lib.sse_state_transfer.argtypes = [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int]
    lib.sse_state_sync.argtypes = [ct.c_void_p]
    lib.sse_state_inject.argtypes = [ct.c_void_p, ct.c_int, ct.c_int]
    lib.sse_state_set_f32.argtypes = [ct.c_void_p, ct.c_int, ct.c_void_p]
    lib.sse_state_get_f32.argtypes = [ct.c_void_p, ct.c_int, ct.c_void_p]
    lib.sse_tune.argtypes = [ct.c_void_p, ct.POINTER(Params), ct.c_int, ct.POINTER(Tuning)]
    lib.sse_server_submit.argtypes = [ct.c_void_p, ct.c_void_p, ct.POINTER(Params), ct.c_void_p,
                                      ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int,
                                      ct.c_double, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p,
                                      ct.c_void_p, ct.POINTER(ct.c_int64)]
    lib.sse_server_query.argtypes = [ct.c_void_p, ct.c_int64, ct.POINTER(RequestInfo)]
    lib.sse_server_wait.argtypes = [ct.c_void_p, ct.c_int64, ct.c_double,
                                    ct.POINTER(RequestInfo)]
    lib.sse_server_stats.argtypes = [ct.c_void_p, ct.POINTER(ServerInfo)]
    lib.sse_server_release.argtypes = [ct.c_void_p, ct.c_int64]
    lib.sse_server_destroy.argtypes = [ct.c_void_p]
    lib.sse_server_destroy.restype = None
    lib.sse_strerror.argtypes = [ct.c_int]
    lib.sse_strerror.restype = ct.c_char_p
    _lib = lib
    return lib


def _check(rc, what):
    if rc != SSE_OK:
        raise SSEError(rc, what)


class Mesh:
    """Device copy of a TRiSK mesh (any object with the mesh.Mesh attributes)."""

    def __init__(self, mesh, nLayers: int, rest_frac=None, max_level=None, rest_thickness=None):
        """max_level [C] / rest_thickness [C, L]: partial bottom cells."""
        self.lib = load()
        self.L = int(nLayers)
        self.nCells, self.nEdges, self.nVertices = int(mesh.nCells), int(mesh.nEdges), int(
            mesh.nVertices)
        keep = []

        def ia(x):
            a = np.ascontiguousarray(x, dtype=np.int32)
            keep.append(a)
            return a.ctypes.data_as(_ip)

        def da(x):
            a = np.ascontiguousarray(x, dtype=np.float64)
            keep.append(a)
            return a.ctypes.data_as(_dp)

        rf = np.full(self.L, 1.0 / self.L) if rest_frac is None else rest_frac
        self.desc = MeshDesc(self.nCells, self.nEdges, self.nVertices, int(mesh.maxEdges),
                             int(mesh.maxEdges2), self.L, ia(mesh.cellsOnEdge),
                             ia(mesh.verticesOnEdge), ia(mesh.nEdgesOnCell),
                             ia(mesh.edgesOnCell), ia(mesh.cellsOnVertex),
                             ia(mesh.edgesOnVertex), ia(mesh.nEdgesOnEdge),
                             ia(mesh.edgesOnEdge), da(mesh.weightsOnEdge), da(mesh.dcEdge),
                             da(mesh.dvEdge), da(mesh.areaCell), da(mesh.areaTriangle),
                             da(mesh.kiteAreasOnVertex), da(mesh.fEdge), da(mesh.fVertex),
                             da(mesh.bottomDepth), da(rf),
                             None if max_level is None else ia(max_level),
                             None if rest_thickness is None else da(rest_thickness))
        self._keep = keep
        h = ct.c_void_p()
        _check(self.lib.sse_mesh_create(ct.byref(self.desc), ct.byref(h)), "sse_mesh_create")
        self.handle = h

    def close(self):
        if self.handle:
            self.lib.sse_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def barotropic_substep_noalloc(mesh: Mesh, order: int, dt: float, M: int, g: float,
                               ubar_in: int, zeta_in: int, G: int, ubar_out: int, Fzeta_out: int,
                               zeta_out: int = 0, stream: int = 0):
    """Allocation-free sub-cycle on caller-owned device arrays (raw pointers)."""
    lib = load()
    _check(lib.sse_barotropic_substep_noalloc(mesh.handle, int(order), float(dt), int(M),
                                              float(g), ct.c_void_p(ubar_in),
                                              ct.c_void_p(zeta_in), ct.c_void_p(G),
                                              ct.c_void_p(ubar_out), ct.c_void_p(Fzeta_out),
                                              ct.c_void_p(zeta_out or 0),
                                              ct.c_void_p(stream or 0)),
           "sse_barotropic_substep_noalloc")


def step_batch(states, order: int, dts, Ms, n_steps: int, stream=None):
    """sse_step_batch: n_steps large steps of every state, in lock-step, the
    3-D kernels of all states in one launch per kernel and stage on `stream`."""
    n = len(states)
    hs = (ct.c_void_p * n)(*[st.handle.value if hasattr(st.handle, "value") else st.handle
                             for st in states])
    d = (ct.c_double * n)(*[float(x) for x in dts])
    m = (ct.c_int32 * n)(*[int(x) for x in Ms])
    _check(load().sse_step_batch(hs, n, int(order), d, m, int(n_steps), ct.c_void_p(stream or 0)),
           "sse_step_batch")


def fma_rate(precision="fp64") -> float:
    """sse_probe_fma_rate: the measured FMA rate of the current GPU (TFLOP/s)."""
    x = ct.c_double()
    prec = {"fp64": FP64, "mixed": MIXED}[precision]
    _check(load().sse_probe_fma_rate(prec, ct.byref(x)), "sse_probe_fma_rate")
    return x.value


def make_params(params: dict, precision="fp64") -> Params:
    q = dict(params)
    recon = q.get("recon", "consistent")
    recon = RECON[recon] if isinstance(recon, str) else int(recon)
    prec = {"fp64": FP64, "mixed": MIXED}[precision] if isinstance(precision, str) else int(
        precision)
    options = OPT_VMIX if q.get("vmix") else 0
    return Params(prec, recon, int(q.get("nTracers", 1)), options, *[float(q.get(n, d)) for n, d in (
        ("g", 9.80616), ("rho0", 1000.0), ("nu_h", 0.0), ("nu_v", 0.0), ("kappa_h", 0.0),
        ("kappa_v", 0.0), ("c_drag", 0.0), ("eos_rho_ref", 1000.0), ("eos_alpha", 0.2),
        ("eos_beta", 0.8), ("eos_T_ref", 10.0), ("eos_S_ref", 35.0), ("nu_4", 0.0))])


class State:
    """A model state on the GPU (the library owns its device memory)."""

    def __init__(self, mesh: Mesh, params: dict, precision="fp64", stream=None,
                 patch_cells: int = 0, bcl_patch_cells: int = 0):
        self.lib = load()
        self.mesh = mesh
        self.params = make_params(params, precision)
        self.nT = self.params.nTracers
        h = ct.c_void_p()
        t = Tuning(int(patch_cells), int(bcl_patch_cells))
        _check(self.lib.sse_state_create_ex(mesh.handle, ct.byref(self.params), ct.byref(t),
                                             ct.c_void_p(stream or 0), ct.byref(h)),
               "sse_state_create_ex")
        self.handle = h
        ws = params.get("windStress")
        if ws is not None:
            self.set("wind", ws)

    @classmethod
    def init(cls, mesh: Mesh, params: dict, precision, u, h, tr, stream=None):
        """sse_state_init: a state made and filled (u, h, tracers, wind) in one call."""
        self = cls.__new__(cls)
        self.lib = load()
        self.mesh = mesh
        self.params = make_params(params, precision)
        self.nT = self.params.nTracers
        u = np.ascontiguousarray(u, dtype=np.float64)
        h = np.ascontiguousarray(h, dtype=np.float64)
        tr = np.ascontiguousarray(tr, dtype=np.float64)
        ws = params.get("windStress")
        ws = None if ws is None else np.ascontiguousarray(ws, dtype=np.float64)
        hd = ct.c_void_p()
        _check(self.lib.sse_state_init(mesh.handle, ct.byref(self.params), u.ctypes.data,
                                       h.ctypes.data, tr.ctypes.data,
                                       None if ws is None else ws.ctypes.data,
                                       ct.c_void_p(stream or 0), ct.byref(hd)), "sse_state_init")
        self.handle = hd
        return self

    def _shape(self, field):
        E, C, L = self.mesh.nEdges, self.mesh.nCells, self.mesh.L
        return {"u": (E, L), "utilde": (E, L), "h": (C, L), "tracer0": (C, L),
                "tracer1": (C, L), "wind": (E,), "ubar": (E,), "G": (E,), "Fzeta": (E,),
                "zeta": (C,), "zeta_sub": (C,)}[field]

    def set(self, field: str, x):
        a = np.ascontiguousarray(x, dtype=np.float64)
        if a.size != int(np.prod(self._shape(field))):
            raise ValueError(f"{field}: expected shape {self._shape(field)}, got {a.shape}")
        _check(self.lib.sse_state_set(self.handle, FIELD[field], a.ctypes.data), f"set {field}")

    def set_ptr(self, field: str, ptr: int):
        """Set from a host pointer (e.g. a pinned torch tensor's data_ptr())."""
        _check(self.lib.sse_state_set(self.handle, FIELD[field], ct.c_void_p(ptr)),
               f"set {field}")

    def get(self, field: str, out=None) -> np.ndarray:
        if out is None:
            out = np.empty(self._shape(field), dtype=np.float64)
        _check(self.lib.sse_state_get(self.handle, FIELD[field], out.ctypes.data), f"get {field}")
        return out

    def get_ptr(self, field: str, ptr: int):
        _check(self.lib.sse_state_get(self.handle, FIELD[field], ct.c_void_p(ptr)),
               f"get {field}")

    def set_f32(self, field: str, x):
        """FP32 host transfer (u, utilde, ubar, G, tracers only)."""
        a = np.ascontiguousarray(x, dtype=np.float32)
        if a.size != int(np.prod(self._shape(field))):
            raise ValueError(f"{field}: expected shape {self._shape(field)}, got {a.shape}")
        _check(self.lib.sse_state_set_f32(self.handle, FIELD[field], a.ctypes.data),
               f"set_f32 {field}")

    def get_f32(self, field: str, out=None) -> np.ndarray:
        if out is None:
            out = np.empty(self._shape(field), dtype=np.float32)
        _check(self.lib.sse_state_get_f32(self.handle, FIELD[field], out.ctypes.data),
               f"get_f32 {field}")
        return out

    def set_ptr_f32(self, field: str, ptr: int):
        _check(self.lib.sse_state_set_f32(self.handle, FIELD[field], ct.c_void_p(ptr)),
               f"set_f32 {field}")

    def get_ptr_f32(self, field: str, ptr: int):
        _check(self.lib.sse_state_get_f32(self.handle, FIELD[field], ct.c_void_p(ptr)),
               f"get_f32 {field}")

    def transfer_ptr(self, field: str, ptr: int, get: bool, f32: bool = False,
                     asynchronous: bool = False):
        """sse_state_transfer on a host pointer; with asynchronous=True the
        array is read or written in stream order (see sync())."""
        flags = (1 if get else 0) | (2 if f32 else 0) | (4 if asynchronous else 0)
        _check(self.lib.sse_state_transfer(self.handle, FIELD[field], ct.c_void_p(ptr), flags),
               f"transfer {field}")

    def sync(self):
        _check(self.lib.sse_state_sync(self.handle), "sse_state_sync")

    def load_state(self, u, h, tr):
        self.set("u", u)
        self.set("h", h)
        tr = np.asarray(tr)
        for t in range(self.nT):
            self.set(f"tracer{t}", tr[t])

    def read_state(self):
        tr = np.stack([self.get(f"tracer{t}") for t in range(self.nT)])
        return self.get("u"), self.get("h"), tr

    def step(self, order: int, dt: float, M: int, n_steps: int = 1):
        _check(self.lib.sse_step(self.handle, int(order), float(dt), int(M), int(n_steps)),
               "sse_step")

    def baroclinic_feuler(self, dt: float):
        _check(self.lib.sse_baroclinic_feuler(self.handle, float(dt)), "sse_baroclinic_feuler")

    def barotropic_substep(self, order: int, dt: float, M: int):
        _check(self.lib.sse_barotropic_substep(self.handle, int(order), float(dt), int(M)),
               "sse_barotropic_substep")

    def diagnostics(self, check=True) -> dict:
        d = Diag()
        rc = self.lib.sse_diagnostics(self.handle, ct.byref(d))
        if check:
            _check(rc, "sse_diagnostics")
        return dict(volume=d.volume, tracer_content=(d.tracer_content[0], d.tracer_content[1]),
                    kinetic_energy=d.kinetic_energy, max_speed=d.max_speed,
                    min_thickness=d.min_thickness, zeta_min=d.zeta_min, zeta_max=d.zeta_max,
                    step=d.step, nonfinite=bool(d.nonfinite), rc=rc)

    def profile(self, enable: bool):
        _check(self.lib.sse_profile(self.handle, 1 if enable else 0), "sse_profile")

    def profile_read(self) -> dict:
        ms = np.zeros(len(KERNEL_CLASSES))
        n = np.zeros(len(KERNEL_CLASSES), dtype=np.int32)
        _check(self.lib.sse_profile_read(self.handle, ms.ctypes.data, n.ctypes.data),
               "sse_profile_read")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_CLASSES)}

    def patches(self) -> int:
        n = ct.c_int()
        _check(self.lib.sse_state_patches(self.handle, ct.byref(n)), "sse_state_patches")
        return int(n.value)

    def subcycle_shape(self):
        """(threads per patch, tensor memory used) of the tiled sub-cycle."""
        th, tm = ct.c_int(), ct.c_int()
        _check(self.lib.sse_state_subcycle_shape(self.handle, ct.byref(th), ct.byref(tm)),
               "sse_state_subcycle_shape")
        return int(th.value), bool(tm.value)

    def inject_barrier_stall(self, on: bool):
        """Test hook: every grid-barrier wait of the sub-cycle runs out its
        bounded budget while on (sse_state_inject)."""
        _check(self.lib.sse_state_inject(self.handle, 1, 1 if on else 0), "sse_state_inject")

    def graphs(self) -> int:
        n = ct.c_int()
        _check(self.lib.sse_state_graphs(self.handle, ct.byref(n)), "sse_state_graphs")
        return int(n.value)

    def kernels_per_step(self, order: int) -> int:
        return int(self.lib.sse_kernels_per_step(self.handle, int(order)))

    def close(self):
        if self.handle:
            self.lib.sse_state_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def footprint(mesh: Mesh, params: dict, precision="fp64", patch_cells: int = 0,
              bcl_patch_cells: int = 0) -> int:
    """Device bytes sse_state_create would allocate for this mesh and parameters."""
    lib = load()
    prm = make_params(params, precision)
    out = ct.c_size_t()
    t = Tuning(int(patch_cells), int(bcl_patch_cells))
    _check(lib.sse_state_footprint_ex(mesh.handle, ct.byref(prm), ct.byref(t), ct.byref(out)),
           "sse_state_footprint_ex")
    return int(out.value)


def tune_shapes(mesh: Mesh, params: dict, precision="mixed", objective="throughput") -> dict:
    """Autotuned launch shapes (sse_tune): the tiled sub-cycle's and the fused
    baroclinic kernel's patch sizes."""
    lib = load()
    prm = make_params(params, precision)
    t = Tuning()
    _check(lib.sse_tune(mesh.handle, ct.byref(prm), TUNE[objective], ct.byref(t)), "sse_tune")
    return {"patch_cells": int(t.patch_cells), "bcl_patch_cells": int(t.bcl_patch_cells)}


def tune(mesh: Mesh, params: dict, precision="mixed", objective="throughput") -> int:
    """Autotuned patch size of the tiled sub-cycle (sse_tune)."""
    return tune_shapes(mesh, params, precision, objective)["patch_cells"]


STATUS = {0: "done", 1: "pending", 2: "active"}


class Request:
    """A submitted solve: the output arrays fill in when it is done."""

    def __init__(self, server, rid, u_out, h_out, tr_out, keep):
        self.server, self.id = server, rid
        self.u, self.h, self.tr = u_out, h_out, tr_out
        self._keep = keep

    def info(self) -> dict:
        inf = RequestInfo()
        _check(self.server.lib.sse_server_query(self.server.handle, self.id, ct.byref(inf)),
               "sse_server_query")
        return _info(inf)

    def wait(self, timeout: float = -1.0) -> dict:
        inf = RequestInfo()
        rc = self.server.lib.sse_server_wait(self.server.handle, self.id, float(timeout),
                                             ct.byref(inf))
        if rc not in (0, -8):
            _check(rc, "sse_server_wait")
        out = _info(inf)
        if out["status"] not in ("pending", "active"):
            self.server._bufs.pop(self.id, None)
        return out

    def release(self):
        """Drop the finished request's record in the server."""
        _check(self.server.lib.sse_server_release(self.server.handle, self.id),
               "sse_server_release")


def _info(inf) -> dict:
    st = int(inf.status)
    return {"id": int(inf.id), "status": STATUS.get(st, st), "steps_done": int(inf.steps_done),
            "t_submit": inf.t_submit, "t_admit": inf.t_admit, "t_done": inf.t_done,
            "footprint": int(inf.footprint)}


class Server:
    """Continuous-batching request runtime (sse_server_*): requests are admitted
    in arrival order while their footprint fits `hbm_budget` bytes and at most
    `max_active` run; their steps overlap on the device."""

    def __init__(self, hbm_budget: int, max_active: int = 64, steps_per_launch: int = 1,
                 device: int = 0, tune=None, packed: bool = False):
        """packed: the active requests of one precision and order advance in
        rounds, all of them in one sse_step_batch call (SSE_SERVER_PACKED)."""
        self.lib = load()
        h = ct.c_void_p()
        obj = -1 if tune is None else TUNE[tune]
        _check(self.lib.sse_server_create_ex(int(device), int(hbm_budget), int(max_active),
                                             int(steps_per_launch), obj, 1 if packed else 0,
                                             ct.byref(h)),
               "sse_server_create_ex")
        self.handle = h
        self._bufs = {}   # output arrays the worker may still write, by request id

    def submit(self, mesh: Mesh, params: dict, precision, u, h, tr, order: int, dt: float,
               M: int, n_steps: int) -> Request:
        prm = make_params(params, precision)
        u = np.ascontiguousarray(u, dtype=np.float64)
        h = np.ascontiguousarray(h, dtype=np.float64)
        tr = np.ascontiguousarray(tr, dtype=np.float64)
        uo, ho, to = np.empty_like(u), np.empty_like(h), np.empty_like(tr)
        ws = params.get("windStress")
        ws = None if ws is None else np.ascontiguousarray(ws, dtype=np.float64)
        rid = ct.c_int64()
        _check(self.lib.sse_server_submit(self.handle, mesh.handle, ct.byref(prm),
                                          u.ctypes.data, h.ctypes.data, tr.ctypes.data,
                                          None if ws is None else ws.ctypes.data,
                                          int(order), float(dt), int(M), int(n_steps),
                                          uo.ctypes.data, ho.ctypes.data, to.ctypes.data,
                                          ct.byref(rid)), "sse_server_submit")
        self._bufs[int(rid.value)] = (uo, ho, to, mesh)
        return Request(self, int(rid.value), uo, ho, to, (mesh,))

    def stats(self) -> dict:
        inf = ServerInfo()
        _check(self.lib.sse_server_stats(self.handle, ct.byref(inf)), "sse_server_stats")
        return {k: int(getattr(inf, k)) for k in ("pending", "active", "max_active_seen",
                                                  "used_bytes", "peak_bytes", "budget_bytes")}

    def close(self):
        if self.handle:
            self.lib.sse_server_destroy(self.handle)   # admitted requests finish first
            self.handle = None
            self._bufs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
