"""Python binding of libpff (B300 / sm_103a phase-field fracture step).

Argument marshalling only: every step of the method runs in the CUDA
kernels of libpff.so, reached through its C ABI (include/pff.h).  PyTorch
supplies device memory and streams.  Importing this package fails loudly if
the library has not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpff.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libpff.so is not built ({LIB_PATH}); run "
                      "`python paper_2606_23458_b300/build.py` or __graft_entry__.build()")

_lib = C.CDLL(LIB_PATH)

PFF_OK, PFF_ERR_ARG, PFF_ERR_MESH, PFF_ERR_CUDA, PFF_ERR_OOM = 0, 1, 2, 3, 4
PFF_ERR_NOT_CONVERGED, PFF_ERR_TIMEOUT, PFF_ERR_NONFINITE = 5, 6, 7
PFF_AT1, PFF_AT2 = 1, 2
PFF_SPLIT_SPECTRAL, PFF_SPLIT_AMOR, PFF_SPLIT_ISO = 0, 1, 2
PFF_FP64, PFF_FP32_MIXED = 0, 1
PFF_LOOP_GRAPH, PFF_LOOP_HOST = 0, 1
PFF_CG_AUTO, PFF_CG_PHASES, PFF_CG_PERSISTENT, PFF_CG_TEST_TIMEOUT = 0, 1, 2, 3
PFF_CG_STAGED, PFF_CG_FUSED, PFF_CG_FUSED_STAGED, PFF_CG_RESIDENT = 4, 5, 6, 7
CG_KINDS = {PFF_CG_AUTO: "auto", PFF_CG_PHASES: "phases", PFF_CG_PERSISTENT: "persistent",
            PFF_CG_STAGED: "staged", PFF_CG_FUSED: "fused", PFF_CG_FUSED_STAGED: "fused_staged",
            PFF_CG_RESIDENT: "resident"}
CG_FAMILIES = ("phases", "persistent", "staged", "fused", "fused_staged", "resident")

MODELS = {"AT1": PFF_AT1, "AT2": PFF_AT2}
SPLITS = {"spectral": PFF_SPLIT_SPECTRAL, "amor": PFF_SPLIT_AMOR, "iso": PFF_SPLIT_ISO}
PFF_PLANE_STRAIN, PFF_PLANE_STRESS = 0, 1
PFF_OP_ELEMENT, PFF_OP_MERGED = 0, 1
OPERATORS = {"element": PFF_OP_ELEMENT, "merged": PFF_OP_MERGED}
PFF_QS_KRYLOV_FP32, PFF_QS_KRYLOV_MESH = 0, 1
PLANES = {"strain": PFF_PLANE_STRAIN, "stress": PFF_PLANE_STRESS}
PRECISIONS = {"fp64": PFF_FP64, "fp32": PFF_FP32_MIXED}


class PffError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"pff status {status}: {msg}")
        self.status = status


class pff_material(C.Structure):
    _fields_ = [("E", C.c_double), ("nu", C.c_double), ("rho", C.c_double),
                ("Gc", C.c_double), ("l0", C.c_double), ("eta", C.c_double),
                ("model", C.c_int32), ("split", C.c_int32), ("plane", C.c_int32),
                ("reserved", C.c_int32)]


class pff_options(C.Structure):
    _fields_ = [("cg_tol", C.c_double), ("cg_max_it", C.c_int32),
                ("max_restarts", C.c_int32), ("t_ramp", C.c_double),
                ("energy_every", C.c_int32), ("ckpt_every", C.c_int32),
                ("block", C.c_int32), ("loop_mode", C.c_int32), ("variant", C.c_int32),
                ("cg_kernel", C.c_int32), ("damage_every", C.c_int32), ("fuse", C.c_int32)]


class pff_qs_options(C.Structure):
    _fields_ = [("newton_tol", C.c_double), ("newton_max", C.c_int32), ("krylov", C.c_int32),
                ("eta_min", C.c_double), ("eta_max", C.c_double), ("cg_max_it", C.c_int32),
                ("pad", C.c_int32)]


class pff_plate(C.Structure):
    _fields_ = [("N", C.c_int64), ("xy", C.c_void_p), ("Ne", C.c_int64), ("tri", C.c_void_p),
                ("notch", C.c_void_p), ("M", C.c_int64), ("tedges", C.c_void_p),
                ("tvec", C.c_void_p), ("mat", pff_material)]


class pff_state(C.Structure):
    _fields_ = [("u", C.c_void_p), ("v", C.c_void_p), ("a", C.c_void_p),
                ("d", C.c_void_p), ("H", C.c_void_p)]


_P = C.c_void_p
_sig = {
    "pff_mesh_create": [C.c_int64, _P, C.c_int64, _P, _P, C.c_int64, _P, _P, C.c_int32,
                        C.POINTER(C.c_void_p)],
    "pff_mesh_destroy": [_P],
    "pff_mesh_set_material": [_P, C.POINTER(pff_material), C.c_double, C.POINTER(C.c_double)],
    "pff_mesh_info": [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_double),
                      C.POINTER(C.c_int32)],
    "pff_mesh_get_csr": [_P, _P, _P],
    "pff_mesh_get_geometry": [_P, _P, _P, _P, _P],
    "pff_step_explicit": [_P, C.POINTER(pff_state), C.c_double, C.c_double,
                          C.POINTER(pff_options), _P],
    "pff_damage_solve": [_P, _P, _P, _P, C.POINTER(pff_options), C.POINTER(C.c_int32),
                         C.POINTER(C.c_double), C.POINTER(C.c_int32), _P],
    "pff_run_host": [_P, C.POINTER(pff_state), C.POINTER(pff_state), C.c_int64, C.c_int64, C.c_double,
                     C.POINTER(pff_options), _P, _P],
    "pff_run": [_P, C.POINTER(pff_state), C.c_int64, C.c_int64, C.c_double,
                C.POINTER(pff_options), _P, _P, _P],
    "pff_sync_status": [_P, _P],
    "pff_energies": [_P, C.POINTER(pff_state), _P, _P],
    "pff_profile_kernels": [_P, C.POINTER(pff_state), C.c_double, C.POINTER(pff_options),
                            C.c_int32, _P, _P],
    "pff_mesh_schedule": [_P, _P, _P],
    "pff_mesh_fused_schedule": [_P, _P, _P],
    "pff_mesh_cg_choice": [_P, _P, _P, _P],
    "pff_mesh_resident_forms": [_P, _P],
    "pff_subcycling_limit": [C.POINTER(pff_material), C.POINTER(C.c_double), C.POINTER(C.c_int32)],
    "pff_ckpt_create": [_P, C.c_int64, C.c_int32, C.POINTER(C.c_void_p)],
    "pff_ckpt_create_policy": [_P, C.c_int64, C.c_int32, C.c_int32, C.POINTER(C.c_void_p)],
    "pff_ckpt_destroy": [_P],
    "pff_ckpt_stats": [_P, C.POINTER(C.c_int64)],
    "pff_run_ckpt": [_P, C.POINTER(pff_state), C.c_int64, C.c_int64, C.c_double,
                     C.POINTER(pff_options), _P, _P, _P],
    "pff_backward": [_P, _P, _P, C.POINTER(pff_options), C.POINTER(C.c_double), _P],
    "pff_backward_field": [_P, _P, _P, C.POINTER(pff_options), C.POINTER(C.c_double), _P, _P],
    "pff_mesh_set_gc_field": [_P, _P],
    "pff_qs_run": [_P, C.POINTER(pff_state), _P, C.c_int64, C.c_int32, C.c_double,
                   C.POINTER(pff_qs_options), C.POINTER(pff_options), _P, _P, _P],
    "pff_batch_create": [C.c_int32, _P, C.c_int32, C.c_double, C.POINTER(C.c_void_p)],
    "pff_batch_destroy": [_P],
    "pff_batch_size": [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
    "pff_batch_plate_info": [_P, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                             C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_double)],
    "pff_batch_run": [_P, C.POINTER(pff_state), C.c_int64, C.c_int64, C.POINTER(pff_options), _P, _P],
    "pff_mesh_set_operator": [_P, C.c_int32],
    "pff_mesh_get_operator": [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
    "pff_batch_set_operator": [_P, C.c_int32],
    "pff_batch_tuning": [_P, _P, _P],
    "pff_damage_solve_noalloc": [_P, _P, _P, _P, C.POINTER(pff_options), C.POINTER(C.c_int32),
                                 C.POINTER(C.c_double), C.POINTER(C.c_int32), _P],
}
for _name, _args in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = None if _name in ("pff_mesh_destroy", "pff_ckpt_destroy", "pff_batch_destroy") else C.c_int
_lib.pff_last_error.restype = C.c_char_p
_lib.pff_version.restype = C.c_char_p


def _check(st):
    if st != PFF_OK:
        raise PffError(st, _lib.pff_last_error().decode())
    return st


def version():
    return _lib.pff_version().decode()


def _np(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def _hp(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def options(cg_tol=1e-8, cg_max_it=10000, max_restarts=50, t_ramp=0.05e-6, energy_every=0,
            ckpt_every=25, block=0, loop_mode=PFF_LOOP_GRAPH, variant=0, cg_kernel=PFF_CG_AUTO,
            damage_every=0, fuse=0):
    """pff_options; fuse: 0 autotuned, 1 separate force and right-hand-side
    kernels, 2 the fused kernel."""
    return pff_options(cg_tol, cg_max_it, max_restarts, t_ramp, energy_every, ckpt_every,
                       block, loop_mode, variant, cg_kernel, damage_every, fuse)


def qs_options(newton_tol=1e-8, newton_max=25, krylov="fp32", eta_min=None, eta_max=0.5,
               cg_max_it=100000):
    """Options of the quasi-static loop (pff_qs_options).  krylov: "fp32"
    (tangent CG in FP32; mixed-precision refinement under an FP64 mesh) or
    "mesh" (the mesh's precision).  eta_min None: 1e-4 with FP32 CG, else 0."""
    k = {"fp32": PFF_QS_KRYLOV_FP32, "mesh": PFF_QS_KRYLOV_MESH}[krylov]
    if eta_min is None:
        eta_min = 1e-4 if k == PFF_QS_KRYLOV_FP32 else 0.0
    return pff_qs_options(newton_tol, newton_max, k, eta_min, eta_max, cg_max_it, 0)


def subcycling_limit(mat):
    """(c_p / (0.6 c_R), N_max) for a material dict: the admissible damage
    subcycling factor (pff_subcycling_limit)."""
    r = C.c_double()
    n = C.c_int32()
    _check(_lib.pff_subcycling_limit(C.byref(material(mat)), C.byref(r), C.byref(n)))
    return r.value, n.value


def material(mat):
    return pff_material(float(mat["E"]), float(mat["nu"]), float(mat["rho"]), float(mat["Gc"]),
                        float(mat["l0"]), float(mat.get("eta", 1e-7)),
                        MODELS[mat.get("model", "AT2")], SPLITS[mat.get("split", "spectral")],
                        PLANES[mat.get("plane", "strain")], 0)


def _dptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


class Batch:
    """pff_batch: independent plates advanced together (one graph launch per
    step for all plates, per-plate CG convergence).  `plates` is a list of
    (plate dict from pff_synth.plate, material dict)."""

    def __init__(self, plates, precision="fp32", cfl=0.5):
        self._keep = []
        arr = (pff_plate * len(plates))()
        self.notch = []
        for k, (p, mat) in enumerate(plates):
            xy = _np(p["xy"], np.float64); tri = _np(p["tri"], np.int32)
            notch = _np(p["notch"], np.uint8); ed = _np(p["tedges"], np.int32)
            tv = _np(p["tvec"], np.float64)
            self._keep += [xy, tri, notch, ed, tv]
            self.notch.append(notch)
            arr[k] = pff_plate(xy.shape[0], _hp(xy).value, tri.shape[0], _hp(tri).value, _hp(notch).value,
                               ed.shape[0], _hp(ed).value, _hp(tv).value, material(mat))
        h = C.c_void_p()
        _check(_lib.pff_batch_create(len(plates), C.cast(arr, C.c_void_p), PRECISIONS[precision],
                                     float(cfl), C.byref(h)))
        self._h = h
        self.precision = precision
        self.nplates = len(plates)
        N = C.c_int64(); Ne = C.c_int64()
        _check(_lib.pff_batch_size(self._h, C.byref(N), C.byref(Ne)))
        self.N, self.Ne = N.value, Ne.value
        self.info = []
        for k in range(self.nplates):
            a = [C.c_int64() for _ in range(4)]; dt = C.c_double()
            _check(_lib.pff_batch_plate_info(self._h, k, *[C.byref(x) for x in a], C.byref(dt)))
            self.info.append(dict(node0=a[0].value, N=a[1].value, elem0=a[2].value, Ne=a[3].value,
                                  dt=dt.value))

    def close(self):
        if getattr(self, "_h", None):
            _lib.pff_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == "fp64" else torch.float32

    def new_state(self, device="cuda"):
        import torch
        dt = self.dtype
        d = torch.zeros(self.N, dtype=dt, device=device)
        for k, inf in enumerate(self.info):
            d[inf["node0"]:inf["node0"] + inf["N"]] = torch.as_tensor(self.notch[k], device=device).to(dt)
        return dict(u=torch.zeros(self.N, 2, dtype=dt, device=device),
                    v=torch.zeros(self.N, 2, dtype=dt, device=device),
                    a=torch.zeros(self.N, 2, dtype=dt, device=device), d=d,
                    H=torch.zeros(self.Ne, dtype=torch.float64, device=device))

    def plate(self, st, k):
        """Views of plate k's part of a concatenated state."""
        inf = self.info[k]
        n0, n1 = inf["node0"], inf["node0"] + inf["N"]
        e0, e1 = inf["elem0"], inf["elem0"] + inf["Ne"]
        return dict(u=st["u"][n0:n1], v=st["v"][n0:n1], a=st["a"][n0:n1], d=st["d"][n0:n1],
                    H=st["H"][e0:e1])

    def tuning(self):
        """The loop configuration (pff_batch_tuning): gathers in flight of the
        force, right-hand side and CG kernels, the CG loop form ("phases",
        "persistent" or "resident"), whether the autotuner has run, the
        persistent launch's CTAs, and the autotuner's timings in ms."""
        ch = np.zeros(6, np.int32)
        ms = np.zeros((3, 12), np.float32)
        _check(_lib.pff_batch_tuning(self._h, _hp(ch), _hp(ms)))
        return dict(force_U=int(ch[0]), rhs_U=int(ch[1]), cg=CG_KINDS.get(int(ch[2]), str(int(ch[2]))),
                    cg_U=int(ch[3]), tuned=bool(ch[4]), persistent_ctas=int(ch[5]),
                    ms=dict(force=[float(x) for x in ms[0, :4]], rhs=[float(x) for x in ms[1, :4]],
                            cg_phases=[float(x) for x in ms[2, :4]], cg_persistent=[float(x) for x in ms[2, 4:7]],
                            cg_resident=[float(x) for x in ms[2, 7:11]]))

    def set_operator(self, form):
        """Damage operator form of every plate: "element" (matrix-free, the
        default) or "merged" (pff_batch_set_operator)."""
        _check(_lib.pff_batch_set_operator(self._h, OPERATORS[form]))

    def run(self, st, nsteps, step0=0, opts=None, iters_log=None, stream=None):
        s = pff_state(st["u"].data_ptr(), st["v"].data_ptr(), st["a"].data_ptr(), st["d"].data_ptr(),
                      st["H"].data_ptr())
        o = opts or options()
        _check(_lib.pff_batch_run(self._h, C.byref(s), int(step0), int(nsteps), C.byref(o),
                                  _dptr(iters_log), _stream(stream)))


class Checkpoint:
    """pff_ckpt: the tape of a run of nsteps steps, consumed by Mesh.backward.
    every = 0 tapes every step during the forward (no recompute); every > 0
    keeps checkpoints at segment starts and recomputes each segment in the
    backward: in full ("recompute"), or only its mechanics, the forward
    having taped each step's unclamped damage solution ("damage_tape")."""

    POLICIES = {"recompute": 0, "damage_tape": 1}

    def __init__(self, mesh, nsteps, every=25, policy="recompute"):
        h = C.c_void_p()
        _check(_lib.pff_ckpt_create_policy(mesh._h, int(nsteps), int(every), self.POLICIES[policy],
                                           C.byref(h)))
        self.policy = policy
        self._h = h
        self.mesh = mesh
        self.nsteps = int(nsteps)
        self.every = int(every)

    def adjoint_iters(self):
        n = C.c_int64()
        _check(_lib.pff_ckpt_stats(self._h, C.byref(n)))
        return n.value

    def close(self):
        if getattr(self, "_h", None):
            _lib.pff_ckpt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    """A device mesh (pff_mesh handle) and its material."""

    def __init__(self, xy, tri, notch=None, tedges=None, tvec=None, precision="fp32"):
        xy = _np(xy, np.float64)
        tri = _np(tri, np.int32)
        self.N, self.Ne = xy.shape[0], tri.shape[0]
        notch = None if notch is None else _np(notch, np.uint8)
        if tedges is None:
            tedges, tvec = np.zeros((0, 2), np.int32), np.zeros((0, 2))
        tedges = _np(tedges, np.int32)
        tvec = _np(tvec, np.float64)
        self.precision = precision
        h = C.c_void_p()
        _check(_lib.pff_mesh_create(self.N, _hp(xy), self.Ne, _hp(tri), _hp(notch),
                                    tedges.shape[0], _hp(tedges), _hp(tvec),
                                    PRECISIONS[precision], C.byref(h)))
        self._h = h
        self.notch = np.zeros(self.N, np.uint8) if notch is None else notch
        self.mat = None
        self.dt = None

    @classmethod
    def from_plate(cls, p, precision="fp32"):
        return cls(p["xy"], p["tri"], p["notch"], p["tedges"], p["tvec"], precision)

    def close(self):
        if getattr(self, "_h", None):
            _lib.pff_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == "fp64" else torch.float32

    def set_material(self, mat, cfl=0.5):
        m = material(mat)
        dt = C.c_double()
        _check(_lib.pff_mesh_set_material(self._h, C.byref(m), float(cfl), C.byref(dt)))
        self.mat = dict(mat)
        self.dt = dt.value
        self.cfl = cfl
        return dt.value

    def info(self):
        N = C.c_int64(); Ne = C.c_int64(); h = C.c_double(); p = C.c_int32()
        _check(_lib.pff_mesh_info(self._h, C.byref(N), C.byref(Ne), C.byref(h), C.byref(p)))
        return dict(N=N.value, Ne=Ne.value, hmin=h.value, precision=p.value)

    def csr(self):
        ptr = np.zeros(self.N + 1, np.int32)
        ent = np.zeros(3 * self.Ne, np.int32)
        _check(_lib.pff_mesh_get_csr(self._h, _hp(ptr), _hp(ent)))
        return ptr, ent

    def geometry(self):
        area = np.zeros(self.Ne); grad = np.zeros((self.Ne, 3, 2))
        fext = np.zeros((self.N, 2)); minv = np.zeros(self.N)
        _check(_lib.pff_mesh_get_geometry(self._h, _hp(area), _hp(grad), _hp(fext),
                                          _hp(minv) if self.mat is not None else None))
        return area, grad, fext, minv

    def new_state(self, device="cuda"):
        import torch
        dt = self.dtype
        d = torch.as_tensor(self.notch, device=device).to(dt)
        return dict(u=torch.zeros(self.N, 2, dtype=dt, device=device),
                    v=torch.zeros(self.N, 2, dtype=dt, device=device),
                    a=torch.zeros(self.N, 2, dtype=dt, device=device),
                    d=d.contiguous(),
                    H=torch.zeros(self.Ne, dtype=torch.float64, device=device))

    def _state(self, st):
        for k in ("u", "v", "a", "d"):
            t = st[k]
            assert t.is_cuda and t.is_contiguous() and t.dtype == self.dtype, k
        assert st["H"].dtype.is_floating_point and st["H"].element_size() == 8
        return pff_state(st["u"].data_ptr(), st["v"].data_ptr(), st["a"].data_ptr(),
                         st["d"].data_ptr(), st["H"].data_ptr())

    def run_host(self, host, st, nsteps, step0=0, dt=None, opts=None, iters_log=None, stream=None):
        """pff_run_host: nsteps steps of the state held in `host` (pinned CPU
        tensors u, v, a, d, H in the mesh precision), with `st` (device
        tensors of the same shapes) as the device workspace; each step copies
        the state in and back out."""
        for k in ("u", "v", "a", "d", "H"):
            t = host[k]
            assert not t.is_cuda and t.is_pinned() and t.is_contiguous(), k
            assert t.shape == st[k].shape and t.dtype == st[k].dtype, k
        h = pff_state(host["u"].data_ptr(), host["v"].data_ptr(), host["a"].data_ptr(),
                      host["d"].data_ptr(), host["H"].data_ptr())
        s = self._state(st)
        o = opts or options()
        _check(_lib.pff_run_host(self._h, C.byref(h), C.byref(s), int(step0), int(nsteps),
                                 float(dt or self.dt), C.byref(o), _dptr(iters_log), _stream(stream)))

    def step_explicit(self, st, t_next, dt=None, opts=None, stream=None):
        s = self._state(st)
        o = opts or options()
        _check(_lib.pff_step_explicit(self._h, C.byref(s), float(t_next), float(dt or self.dt),
                                      C.byref(o), _stream(stream)))

    def damage_solve(self, H, dprev, dout, opts=None, stream=None, raise_on_error=True):
        o = opts or options()
        it = C.c_int32(); rel = C.c_double(); rs = C.c_int32()
        st = _lib.pff_damage_solve(self._h, _dptr(H), _dptr(dprev), _dptr(dout), C.byref(o),
                                   C.byref(it), C.byref(rel), C.byref(rs), _stream(stream))
        if raise_on_error:
            _check(st)
        return dict(status=st, iters=it.value, relres=rel.value, restarts=rs.value)

    def damage_solve_noalloc(self, H, dprev, dout, opts=None, stream=None, raise_on_error=True):
        """pff_damage_solve_noalloc: the same solve without any device
        allocation during the call (statically reserved workspace, meshes up
        to 131,072 nodes / 262,144 elements; concurrent calls race)."""
        o = opts or options()
        it = C.c_int32(); rel = C.c_double(); rs = C.c_int32()
        st = _lib.pff_damage_solve_noalloc(self._h, _dptr(H), _dptr(dprev), _dptr(dout), C.byref(o),
                                           C.byref(it), C.byref(rel), C.byref(rs), _stream(stream))
        if raise_on_error:
            _check(st)
        return dict(status=st, iters=it.value, relres=rel.value, restarts=rs.value)

    def run(self, st, nsteps, step0=0, dt=None, opts=None, iters_log=None, energy_log=None,
            stream=None):
        s = self._state(st)
        o = opts or options()
        _check(_lib.pff_run(self._h, C.byref(s), int(step0), int(nsteps), float(dt or self.dt),
                            C.byref(o), _dptr(iters_log), _dptr(energy_log), _stream(stream)))

    def run_ckpt(self, st, ckpt, step0=0, dt=None, opts=None, iters_log=None, stream=None):
        s = self._state(st)
        o = opts or options()
        _check(_lib.pff_run_ckpt(self._h, C.byref(s), int(step0), ckpt.nsteps, float(dt or self.dt),
                                 C.byref(o), ckpt._h, _dptr(iters_log), _stream(stream)))

    def backward(self, ckpt, dL_dd, opts=None, stream=None):
        """dL/dGc (float) for the upstream gradient dL/dd at the final step."""
        assert dL_dd.is_cuda and dL_dd.dtype == self.dtype and dL_dd.is_contiguous()
        o = opts or options()
        g = C.c_double()
        _check(_lib.pff_backward(self._h, ckpt._h, _dptr(dL_dd), C.byref(o), C.byref(g),
                                 _stream(stream)))
        return g.value

    def backward_field(self, ckpt, dL_dd, opts=None, stream=None):
        """(dL/dGc, dL/dGc_e per element as a float64 device tensor)."""
        import torch
        assert dL_dd.is_cuda and dL_dd.dtype == self.dtype and dL_dd.is_contiguous()
        o = opts or options()
        g = C.c_double()
        ge = torch.empty(self.Ne, dtype=torch.float64, device=dL_dd.device)
        _check(_lib.pff_backward_field(self._h, ckpt._h, _dptr(dL_dd), C.byref(o), C.byref(g),
                                       _dptr(ge), _stream(stream)))
        return g.value, ge

    def qs_run(self, st, bc, nincr, du, incr0=0, qopts=None, opts=None, stream=None, **kw):
        """Quasi-static staggered increments (pff_qs_run).  bc: N uint8
        flags (1 fix u_x, 2 fix u_y, 4 loaded: u_y = U).  qopts: a
        qs_options(...) (or its keywords in kw).  Returns dict(reaction
        (nincr,), iters (nincr, 3): Newton, mechanics CG, damage CG)."""
        s = self._state(st)
        q = qopts if qopts is not None else qs_options(**kw)
        o = opts or options()
        b = _np(bc, np.uint8)
        assert b.shape == (self.N,)
        reac = np.zeros(nincr)
        it = np.zeros((nincr, 3), np.int32)
        _check(_lib.pff_qs_run(self._h, C.byref(s), _hp(b), int(incr0), int(nincr), float(du),
                               C.byref(q), C.byref(o), _hp(reac), _hp(it), _stream(stream)))
        return dict(reaction=reac, iters=it)

    def set_operator(self, form):
        """Damage operator form: "element" (matrix-free, the default) or
        "merged" (rows assembled per solve; pff_mesh_set_operator)."""
        _check(_lib.pff_mesh_set_operator(self._h, OPERATORS[form]))

    def operator(self):
        """(form name, whether "merged" is available on this mesh)."""
        f = C.c_int32(); a = C.c_int32()
        _check(_lib.pff_mesh_get_operator(self._h, C.byref(f), C.byref(a), None))
        return {v: k for k, v in OPERATORS.items()}[f.value], bool(a.value)

    def fan_order(self):
        """Whether the element-wise entries are stored in fan order."""
        v = C.c_int32()
        _check(_lib.pff_mesh_get_operator(self._h, None, None, C.byref(v)))
        return bool(v.value)

    def set_gc_field(self, gc):
        """Per-element toughness Gc_e (array of Ne, host), or None for the
        material's uniform Gc."""
        if gc is None:
            _check(_lib.pff_mesh_set_gc_field(self._h, None))
            return
        a = _np(gc, np.float64)
        assert a.shape == (self.Ne,)
        _check(_lib.pff_mesh_set_gc_field(self._h, _hp(a)))

    def sync_status(self, stream=None):
        return _lib.pff_sync_status(self._h, _stream(stream))

    def schedule(self):
        """(variant codes for force, rhs, matvec; autotuner ms per variant)."""
        var = np.zeros(3, np.int32)
        ms = np.zeros((3, 5), np.float32)
        _check(_lib.pff_mesh_schedule(self._h, _hp(var), _hp(ms)))
        names = ("force", "rhs", "matvec")
        return ({n: int(v) for n, v in zip(names, var)},
                {n: [round(float(x), 4) for x in row] for n, row in zip(names, ms)})

    def fused_schedule(self):
        """(variant code of the fused force and right-hand side in use,
        autotuner ms per variant)."""
        var = C.c_int32()
        ms = np.zeros(5, np.float32)
        _check(_lib.pff_mesh_fused_schedule(self._h, C.byref(var), _hp(ms)))
        return var.value, [round(float(x), 4) for x in ms]

    def cg_choice(self):
        """(AT2 CG loop in use: "auto" (not timed yet) / "phases" /
        "persistent" / "staged" / "fused" / "fused_staged" / "resident", its
        variant (gathers in flight, or the resident kernel's CTA shape), and
        {loop: ms of 30 iterations of its best variant})."""
        k = C.c_int32()
        u = C.c_int32()
        ms = np.zeros(len(CG_FAMILIES), np.float32)
        _check(_lib.pff_mesh_cg_choice(self._h, C.byref(k), C.byref(u), _hp(ms)))
        return CG_KINDS[k.value], u.value, {n: float(x) for n, x in zip(CG_FAMILIES, ms)}

    RESIDENT_FORMS = {-1: None, 0: "partial", 1: "full"}

    def resident_forms(self):
        """Form of the resident CG loop per CTA shape U = 1..4: None
        (unavailable), "partial" or "full"."""
        f = np.zeros(4, np.int32)
        _check(_lib.pff_mesh_resident_forms(self._h, _hp(f)))
        return [self.RESIDENT_FORMS[int(v)] for v in f]

    KERNELS = ("predict", "force", "rhs", "matvec", "update", "finish", "energies")

    def profile_kernels(self, st, reps=5, opts=None, dt=None, stream=None):
        """Average device ms per launch of each kernel on this data (L2
        flushed before every launch).  Overwrites the state."""
        s = self._state(st)
        o = opts or options()
        out = np.zeros(12)
        _check(_lib.pff_profile_kernels(self._h, C.byref(s), float(dt or self.dt), C.byref(o),
                                        int(reps), _hp(out), _stream(stream)))
        d = dict(zip(self.KERNELS, out[:7].tolist()))
        d["cg_loop"] = float(out[7])          # one persistent CG launch (0: kernel per phase)
        d["cg_loop_iters"] = int(out[8])
        d["cg_loop_family"] = CG_FAMILIES[int(out[9])]
        d["force_rhs"] = float(out[10])        # the fused force and right-hand-side kernel
        d["force_rhs_used"] = bool(out[11])
        return d

    def energies(self, st, stream=None):
        s = self._state(st)
        out = np.zeros(3)
        _check(_lib.pff_energies(self._h, C.byref(s), _hp(out), _stream(stream)))
        return out
