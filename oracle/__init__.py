"""FP64 CPU oracle for the phase-field fracture step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the bench's ``cpu_baseline``
leg may import this package.  It wraps ``pff_oracle.c`` (plain C, fp64, one
element at a time in element-id order) through ctypes and shares no code with
the CUDA library.  Each function cites the passage of the paper it follows
in the C source.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against a closed form, an invariant, brute force or a textbook routine (see
tests/test_oracle_*.py); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pff_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MODELS = {"AT1": 1, "AT2": 2}
SPLITS = {"spectral": 0, "amor": 1, "iso": 2}
PLANES = {"strain": 0, "stress": 1}


def build(force=False):
    """Compile the oracle with gcc (no fast-math, no FMA contraction, so the
    arithmetic is the plain IEEE sequence the source spells out)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off",
                               "-shared", "-fPIC", "-o", _LIB, _SRC, "-lm"])
    return _LIB


class _Mat(C.Structure):
    _fields_ = [("E", C.c_double), ("nu", C.c_double), ("rho", C.c_double),
                ("Gc", C.c_double), ("l0", C.c_double), ("eta", C.c_double),
                ("model", C.c_int32), ("split", C.c_int32),
                ("plane", C.c_int32), ("pad", C.c_int32)]


class _RunOpts(C.Structure):
    _fields_ = [("dt", C.c_double), ("t_ramp", C.c_double), ("tol", C.c_double),
                ("max_it", C.c_int32), ("max_restarts", C.c_int32),
                ("damage_on", C.c_int32), ("energy_every", C.c_int32), ("n_sub", C.c_int32)]


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        _lib.or_mesh_create.restype = P
        _lib.or_mesh_create.argtypes = [C.c_int64, P, C.c_int64, P, P, C.c_int64, P, P, P]
        _lib.or_mesh_free.argtypes = [P]
        _lib.or_mesh_geometry.argtypes = [P, P, P, P, P]
        _lib.or_lumped_mass.argtypes = [P, C.c_double, P]
        _lib.or_csr.argtypes = [P, P, P]
        _lib.or_colour.argtypes = [P, P]
        _lib.or_colour.restype = C.c_int
        _lib.or_stable_dt.argtypes = [P, P, C.c_double]
        _lib.or_stable_dt.restype = C.c_double
        _lib.or_constitutive.argtypes = [P, P, C.c_double, P, P, P, P, P]
        _lib.or_constitutive_tangent.argtypes = [P, P, C.c_double, P, P]
        _lib.or_internal_force.argtypes = [P, P, P, P, P, P]
        _lib.or_ramp.argtypes = [C.c_double, C.c_double]
        _lib.or_ramp.restype = C.c_double
        _lib.or_damage_apply.argtypes = [P, P, P, P, P]
        _lib.or_damage_rhs.argtypes = [P, P, P, P, P]
        _lib.or_damage_solve.argtypes = [P, P, P, P, P, C.c_double, C.c_int, C.c_int,
                                         C.c_int, P, P, P]
        _lib.or_energies.argtypes = [P, P, P, P, P, P, P]
        _lib.or_run.argtypes = [P, P, P, C.c_int64, C.c_int64, P, P, P, P, P, P, P, P, P, P]
        _lib.or_run.restype = C.c_int
        _lib.or_adjoint_gc.argtypes = [P, P, P, C.c_int64, P, P, P, P, P, P, P, P, P]
        _lib.or_adjoint_gc.restype = C.c_int
        _lib.or_elem_adjoint.argtypes = [P, P, P, P, P, P, P, P]
        _lib.or_damage_adjoint_terms.argtypes = [P, P, P, P, P, P, P]
        _lib.or_mesh_set_gc_field.argtypes = [P, P]
        _lib.or_mesh_set_gc_field.restype = None
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def material(mat):
    """ctypes struct from a material dict (E, nu, rho, Gc, l0, eta, model,
    split, plane)."""
    return _Mat(float(mat["E"]), float(mat["nu"]), float(mat["rho"]),
                float(mat["Gc"]), float(mat["l0"]), float(mat.get("eta", 1e-7)),
                MODELS[mat.get("model", "AT2")], SPLITS[mat.get("split", "spectral")],
                PLANES[mat.get("plane", "strain")], 0)


def subcycling_limit(mat):
    """(c_p / (0.6 c_R), N_max = floor of it): the pre-simulation check of the
    damage subcycling factor (Sec. 2.4, sec:subcycling)."""
    m = material(mat)
    r = C.c_double()
    n = C.c_int32()
    _L().or_subcycling_limit(C.byref(m), C.byref(r), C.byref(n))
    return r.value, n.value


def ramp(t, t_ramp):
    """Eq. (smooth_traction_ramp)."""
    return _L().or_ramp(float(t), float(t_ramp))


def constitutive(mat, eps, dbar=0.0):
    """(sigma, sigma+, psi+, psi-, psi) at strain eps = (exx, eyy, exy)."""
    m = material(mat)
    e = _f64(eps, (3,))
    sig = np.zeros(3); sp = np.zeros(3)
    pp = C.c_double(); pm = C.c_double(); ps = C.c_double()
    _L().or_constitutive(C.byref(m), _p(e), float(dbar), _p(sig), _p(sp),
                         C.byref(pp), C.byref(pm), C.byref(ps))
    return sig, sp, pp.value, pm.value, ps.value


def constitutive_tangent(mat, eps, dbar, de):
    m = material(mat)
    e = _f64(eps, (3,)); d = _f64(de, (3,))
    ds = np.zeros(3)
    _L().or_constitutive_tangent(C.byref(m), _p(e), float(dbar), _p(d), _p(ds))
    return ds


class OracleError(RuntimeError):
    pass


class Mesh:
    """Oracle mesh: geometry of Eq. (grad_phi), traction load, notch set."""

    def __init__(self, xy, tri, notch=None, tedges=None, tvec=None):
        self.xy = _f64(xy)
        self.tri = np.ascontiguousarray(np.asarray(tri, dtype=np.int32))
        self.N = self.xy.shape[0]
        self.Ne = self.tri.shape[0]
        self.notch = (np.zeros(self.N, np.uint8) if notch is None
                      else np.ascontiguousarray(np.asarray(notch, dtype=np.uint8)))
        if tedges is None:
            tedges = np.zeros((0, 2), np.int32)
            tvec = np.zeros((0, 2))
        self.tedges = np.ascontiguousarray(np.asarray(tedges, dtype=np.int32))
        self.tvec = _f64(tvec)
        bad = C.c_int64(-1)
        h = _L().or_mesh_create(self.N, _p(self.xy), self.Ne, _p(self.tri), _p(self.notch),
                                self.tedges.shape[0], _p(self.tedges), _p(self.tvec),
                                C.byref(bad))
        if not h:
            raise OracleError(f"invalid mesh (element {bad.value})")
        self._h = C.c_void_p(h)

    @classmethod
    def from_plate(cls, p):
        return cls(p["xy"], p["tri"], p["notch"], p["tedges"], p["tvec"])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.or_mesh_free(h)
            self._h = None

    def geometry(self):
        area = np.zeros(self.Ne); grad = np.zeros((self.Ne, 3, 2))
        fext = np.zeros((self.N, 2)); hmin = C.c_double()
        _L().or_mesh_geometry(self._h, _p(area), _p(grad), _p(fext), C.byref(hmin))
        return area, grad, fext, hmin.value

    def lumped_mass(self, rho):
        m = np.zeros(self.N)
        _L().or_lumped_mass(self._h, float(rho), _p(m))
        return m

    def csr(self):
        ptr = np.zeros(self.N + 1, np.int32); ent = np.zeros(3 * self.Ne, np.int32)
        _L().or_csr(self._h, _p(ptr), _p(ent))
        return ptr, ent

    def colour(self):
        col = np.zeros(self.Ne, np.uint8)
        n = _L().or_colour(self._h, _p(col))
        return col, n

    def stable_dt(self, mat, cfl):
        m = material(mat)
        return _L().or_stable_dt(self._h, C.byref(m), float(cfl))

    def internal_force(self, mat, u, d):
        m = material(mat)
        u = _f64(u, (self.N, 2)); d = _f64(d, (self.N,))
        f = np.zeros((self.N, 2)); pp = np.zeros(self.Ne)
        _L().or_internal_force(self._h, C.byref(m), _p(u), _p(d), _p(f), _p(pp))
        return f, pp

    def damage_apply(self, mat, H, p):
        m = material(mat)
        H = _f64(H, (self.Ne,)); p = _f64(p, (self.N,))
        q = np.zeros(self.N)
        _L().or_damage_apply(self._h, C.byref(m), _p(H), _p(p), _p(q))
        return q

    def damage_rhs(self, mat, H):
        m = material(mat)
        H = _f64(H, (self.Ne,))
        b = np.zeros(self.N); dg = np.zeros(self.N)
        _L().or_damage_rhs(self._h, C.byref(m), _p(H), _p(b), _p(dg))
        return b, dg

    def damage_solve(self, mat, H, dprev, tol=1e-8, max_it=10000, max_restarts=50,
                     forced=-1):
        """Returns (d, info, relres, status, x): info = (iterations, AT2
        natural stop count | AT1 restarts), x = unclamped AT2 solution."""
        m = material(mat)
        H = _f64(H, (self.Ne,)); dp = _f64(dprev, (self.N,))
        d = np.zeros(self.N); x = np.zeros(self.N)
        info = np.zeros(2, np.int32); rel = C.c_double()
        st = _L().or_damage_solve(self._h, C.byref(m), _p(H), _p(dp), _p(d), float(tol),
                                  int(max_it), int(max_restarts), int(forced), _p(info),
                                  C.byref(rel), _p(x))
        return d, info, rel.value, st, x

    def energies(self, mat, u, v, d):
        m = material(mat)
        mass = self.lumped_mass(mat["rho"])
        u = _f64(u, (self.N, 2)); v = _f64(v, (self.N, 2)); d = _f64(d, (self.N,))
        out = np.zeros(3)
        _L().or_energies(self._h, C.byref(m), _p(mass), _p(u), _p(v), _p(d), _p(out))
        return out

    def new_state(self):
        return dict(u=np.zeros((self.N, 2)), v=np.zeros((self.N, 2)),
                    a=np.zeros((self.N, 2)), d=self.notch.astype(np.float64),
                    H=np.zeros(self.Ne))

    def run(self, mat, state, nsteps, dt, n0=0, t_ramp=0.05e-6, tol=1e-8,
            max_it=10000, max_restarts=50, damage_on=True, energy_every=0,
            forced=None, W=0.0, n_sub=1):
        """Runs nsteps staggered steps on `state` (modified in place).
        n_sub > 1: damage solved only after steps n with (n+1) % n_sub == 0
        (subcycling, Sec. 2.4).
        Returns dict(status, iters (nsteps,2), relres, energies (nsteps,4), W)."""
        m = material(mat)
        o = _RunOpts(float(dt), float(t_ramp), float(tol), int(max_it), int(max_restarts),
                     1 if damage_on else 0, int(energy_every), int(n_sub))
        for k in ("u", "v", "a"):
            state[k] = _f64(state[k], (self.N, 2))
        state["d"] = _f64(state["d"], (self.N,))
        state["H"] = _f64(state["H"], (self.Ne,))
        it = np.zeros((nsteps, 2), np.int32)
        rel = np.zeros(nsteps)
        en = np.full((nsteps, 4), np.nan)
        fz = None if forced is None else np.ascontiguousarray(np.asarray(forced, np.int32))
        Wc = C.c_double(W)
        st = _L().or_run(self._h, C.byref(m), C.byref(o), int(n0), int(nsteps),
                         _p(state["u"]), _p(state["v"]), _p(state["a"]), _p(state["d"]),
                         _p(state["H"]), _p(it), _p(rel), _p(en), _p(fz), C.byref(Wc))
        return dict(status=st, iters=it, relres=rel, energies=en, W=Wc.value)

    def set_gc_field(self, gc):
        """Per-element toughness Gc_e (Ne values), or None for the material's
        uniform Gc."""
        self._gcf = None if gc is None else _f64(gc, (self.Ne,))
        _L().or_mesh_set_gc_field(self._h, None if gc is None else _p(self._gcf))

    def adjoint_gc(self, mat, nsteps, dt, dstar, state0=None, t_ramp=0.05e-6,
                   tol=1e-8, max_it=10000, field=False):
        """(loss, dL/dGc, status) for L = mean((d_T - dstar)^2); with
        field=True also dL/dGc_e per element (Ne) as a fourth value."""
        m = material(mat)
        o = _RunOpts(float(dt), float(t_ramp), float(tol), int(max_it), 50, 1, 0, 1)
        s = state0 if state0 is not None else self.new_state()
        u0 = _f64(s["u"], (self.N, 2)); v0 = _f64(s["v"], (self.N, 2))
        a0 = _f64(s["a"], (self.N, 2)); d0 = _f64(s["d"], (self.N,))
        H0 = _f64(s["H"], (self.Ne,)); ds = _f64(dstar, (self.N,))
        L = C.c_double(); g = C.c_double()
        ge = np.zeros(self.Ne) if field else None
        st = _L().or_adjoint_gc(self._h, C.byref(m), C.byref(o), int(nsteps), _p(u0), _p(v0),
                                _p(a0), _p(d0), _p(H0), _p(ds), C.byref(L), C.byref(g),
                                None if ge is None else _p(ge))
        return (L.value, g.value, st, ge) if field else (L.value, g.value, st)

    def elem_adjoint(self, mat, u, d, fbar, psibar=None):
        m = material(mat)
        u = _f64(u, (self.N, 2)); d = _f64(d, (self.N,)); fb = _f64(fbar, (self.N, 2))
        pb = None if psibar is None else _f64(psibar, (self.Ne,))
        ub = np.zeros((self.N, 2)); db = np.zeros(self.N)
        _L().or_elem_adjoint(self._h, C.byref(m), _p(u), _p(d), _p(fb), _p(pb), _p(ub), _p(db))
        return ub, db

    def tangent_apply(self, mat, u, d, p):
        """K_T(u) p: the directional derivative of the internal force at u
        along p with d fixed (Eq. matrix_free_tangent_action); the Hessian of
        sum A_e psi is symmetric, so the element adjoint applies it."""
        return self.elem_adjoint(mat, u, d, p)[0]

    def qs_run(self, mat, state, bc, nincr, du, tol=1e-8, newton_max=25, incr0=0):
        """Quasi-static staggered loop (Sec. 3.5 and the matrix-free tangent
        of Sec. 2.3): per load increment k, the prescribed displacement
        U = (incr0 + k + 1) du is put on the loaded dofs, the mechanics
        f_int(u; d) = 0 on the free dofs is solved by Newton with the
        tangent K_T(u) (assembled here column by column from tangent_apply
        and solved directly, a library step) until ||r_free|| <= tol
        ||f_int||, then H = max(H, psi+(u)) and the damage solve as in a
        dynamic step; the reaction is the sum of f_int,y over the loaded
        nodes before the damage update.
        bc: N flags, 1 = u_x fixed (0), 2 = u_y fixed (0), 4 = loaded node
        (u_y = U; implies 2).  Returns dict(reaction (nincr,), newton
        (nincr,), damage_iters (nincr,), status)."""
        bc = np.asarray(bc, np.uint8)
        fixed = np.zeros((self.N, 2), bool)
        fixed[:, 0] = (bc & 1) != 0
        fixed[:, 1] = (bc & 6) != 0
        loaded = (bc & 4) != 0
        free = np.flatnonzero(~fixed.ravel())
        u = state["u"]; d = state["d"]; H = state["H"]
        out = dict(reaction=np.zeros(nincr), newton=np.zeros(nincr, np.int32),
                   damage_iters=np.zeros(nincr, np.int32), status=0)
        for k in range(nincr):
            U = (incr0 + k + 1) * du
            u[fixed[:, 0], 0] = 0.0
            u[fixed[:, 1], 1] = 0.0
            u[loaded, 1] = U
            for it in range(newton_max + 1):
                f, psip = self.internal_force(mat, u, d)
                r = -f.ravel()[free]
                fn = np.linalg.norm(f)
                if np.linalg.norm(r) <= tol * fn or fn == 0.0:
                    break
                if it == newton_max:
                    out["status"] = 5
                    break
                Kt = np.zeros((free.size, free.size))
                e = np.zeros(2 * self.N)
                for j, dof in enumerate(free):
                    e[dof] = 1.0
                    Kt[:, j] = self.tangent_apply(mat, u, d, e.reshape(self.N, 2)).ravel()[free]
                    e[dof] = 0.0
                step = np.linalg.solve(Kt, r)
                uf = u.ravel()
                uf[free] += step
                u[:] = uf.reshape(self.N, 2)
            out["newton"][k] = it
            out["reaction"][k] = f[loaded, 1].sum()
            np.maximum(H, psip, out=H)
            dn, info, rel, st, _ = self.damage_solve(mat, H, d, tol=tol)
            d[:] = dn
            out["damage_iters"][k] = info[0]
            out["status"] = max(out["status"], st)
        return out

    def damage_adjoint_terms(self, mat, lam, xt):
        m = material(mat)
        lam = _f64(lam, (self.N,)); xt = _f64(xt, (self.N,))
        gc = C.c_double(0.0); Hb = np.zeros(self.Ne)
        _L().or_damage_adjoint_terms(self._h, C.byref(m), _p(lam), _p(xt), C.byref(gc), _p(Hb), None)
        return gc.value, Hb
