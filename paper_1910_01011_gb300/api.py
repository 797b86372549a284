"""Python front end of the C ABI: one Context per bem_ctx.  Arrays are numpy
(host) or torch CUDA tensors (device, complex128, used in place on the
context's stream).  Marshalling only."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import bem_z, check

FP64, FP32, BF16X3, FP64_ASSEMBLED = _lib.PREC_FP64, _lib.PREC_FP32, _lib.PREC_BF16X3, _lib.PREC_FP64_ASSEMBLED
AHAT, PREC, PREC_AHAT = _lib.OP_AHAT, _lib.OP_PREC, _lib.OP_PREC_AHAT


def _z(c) -> bem_z:
    c = complex(c)
    return bem_z(c.real, c.imag)


def _is_torch(a):
    return type(a).__module__.startswith("torch")


class Context:
    def __init__(self, device: int = 0, stream=None, **opts):
        self.lib = _lib.load()
        o = _lib.bem_opts()
        check(self.lib.bem_default_opts(ctypes.byref(o)))
        for k, v in opts.items():
            setattr(o, k, v)
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream(device).cuda_stream
            except ImportError:
                stream = None
        h = ctypes.c_void_p()
        rc = self.lib.bem_create(ctypes.byref(h), device, ctypes.c_void_p(stream or 0), ctypes.byref(o))
        if rc:
            raise _lib.BemError(rc, "bem_create failed")
        self.h = h
        self.device = device
        self.domains = []

    def close(self):
        if getattr(self, "h", None):
            self.lib.bem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        return check(rc, self.h)

    # ---- set-up
    def set_exterior(self, k0, rho0=1.0):
        self._check(self.lib.bem_set_exterior(self.h, _z(k0), float(rho0)))

    def add_domain(self, verts, tris, k, rho):
        v = np.ascontiguousarray(verts, dtype=np.float64)
        t = np.ascontiguousarray(tris, dtype=np.int32)
        i = ctypes.c_int32()
        self._check(self.lib.bem_add_domain(self.h, v.ctypes.data, v.shape[0], t.ctypes.data, t.shape[0], _z(k),
                                            float(rho), ctypes.byref(i)))
        self.domains.append((v.shape[0], t.shape[0]))
        return i.value

    def set_material(self, dom, k, rho):
        self._check(self.lib.bem_set_material(self.h, int(dom), _z(k), float(rho)))

    @classmethod
    def from_scene(cls, scene, device=0, stream=None, **opts):
        c = cls(device, stream, **opts)
        c.set_exterior(scene.k0, scene.rho0)
        for d in scene.domains:
            c.add_domain(d.verts, d.tris, d.k, d.rho)
        return c

    @property
    def n_dofs(self):
        n = ctypes.c_int64()
        self._check(self.lib.bem_num_dofs(self.h, ctypes.byref(n)))
        return n.value

    @property
    def interactions(self):
        n = ctypes.c_int64()
        self._check(self.lib.bem_interaction_count(self.h, ctypes.byref(n)))
        return n.value

    # ---- operators
    def apply(self, x, op=AHAT, precision=FP32, out=None):
        """y = op(x); x (N,) or (n_rhs, N) complex.  numpy -> numpy (host
        copies), torch CUDA -> torch CUDA (device pointers)."""
        N = self.n_dofs
        if _is_torch(x):
            import torch
            assert x.is_cuda and x.dtype == torch.complex128 and x.is_contiguous()
            n_rhs = x.numel() // N
            y = torch.empty_like(x) if out is None else out
            self._check(self.lib.bem_apply(self.h, op, x.data_ptr(), y.data_ptr(), n_rhs, precision, 1))
            return y
        xa = np.ascontiguousarray(x, dtype=np.complex128)
        n_rhs = xa.size // N
        y = np.empty_like(xa) if out is None else out
        self._check(self.lib.bem_apply(self.h, op, xa.ctypes.data, y.ctypes.data, n_rhs, precision, 0))
        return y

    def apply_block(self, test_dom, trial_dom, k, x, precision=FP64):
        """One Calderon block [[-K, V], [W, K']] at wavenumber k, paper order
        x = [phi_i; psi_i] -> [row1; row2] on domain test_dom."""
        xa = np.ascontiguousarray(x, dtype=np.complex128)
        nj = self.domains[test_dom][0]
        y = np.empty(2 * nj, dtype=np.complex128)
        self._check(self.lib.bem_apply_block(self.h, int(test_dom), int(trial_dom), _z(k), xa.ctypes.data,
                                             y.ctypes.data, precision, 0))
        return y

    # ---- incident fields
    def set_plane_wave(self, direction, amp=1.0):
        d = (ctypes.c_double * 3)(*[float(v) for v in direction])
        self._check(self.lib.bem_set_plane_wave(self.h, d, _z(amp)))

    def set_transducer(self, centres, normals, radii, omega_rho0):
        c = np.ascontiguousarray(centres, dtype=np.float64)
        n = np.ascontiguousarray(normals, dtype=np.float64)
        r = np.ascontiguousarray(radii, dtype=np.float64)
        self._check(self.lib.bem_set_transducer(self.h, c.ctypes.data, n.ctypes.data, r.ctypes.data, r.size,
                                                float(omega_rho0)))

    def set_excitations(self, w):
        wa = np.ascontiguousarray(np.atleast_2d(w), dtype=np.complex128)
        self._check(self.lib.bem_set_excitations(self.h, wa.ctypes.data, wa.shape[0]))
        self.n_rhs = wa.shape[0]

    def rhs(self, n_rhs=1):
        b = np.empty(n_rhs * self.n_dofs, dtype=np.complex128)
        self._check(self.lib.bem_rhs(self.h, b.ctypes.data, 0))
        return b.reshape(n_rhs, -1) if n_rhs > 1 else b

    # ---- solve
    def solve(self, **kw):
        o = _lib.bem_solve_opts()
        check(self.lib.bem_default_solve_opts(ctypes.byref(o)))
        for k, v in kw.items():
            setattr(o, k, v)
        r = _lib.bem_solve_report()
        rc = self.lib.bem_solve(self.h, ctypes.byref(o), ctypes.byref(r))
        if rc not in (0, -4):
            self._check(rc)
        return {"iterations": r.iterations, "refinements": r.refinements, "residual": r.residual,
                "seconds": r.seconds, "converged": rc == 0}

    def traces(self, dom, rhs=0):
        nv = self.domains[dom][0]
        d = np.empty(nv, dtype=np.complex128)
        n = np.empty(nv, dtype=np.complex128)
        self._check(self.lib.bem_get_traces(self.h, int(dom), int(rhs), d.ctypes.data, n.ctypes.data, 0))
        return d, n


    def field(self, points, domain_of_point, rhs=0):
        """Total pressure at points (representation formula); domain -1 = exterior."""
        p = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
        d = np.ascontiguousarray(domain_of_point, dtype=np.int32).reshape(-1)
        out = np.empty(p.shape[0], dtype=np.complex128)
        self._check(self.lib.bem_field(self.h, int(rhs), p.ctypes.data, d.ctypes.data, p.shape[0], out.ctypes.data, 0))
        return out

    # ---- measurement
    def profile(self, enable=True):
        self._check(self.lib.bem_profile_enable(self.h, 1 if enable else 0))

    def profile_read(self, reset=True):
        ms = ctypes.c_double()
        nf = ctypes.c_int64()
        nk = ctypes.c_int64()
        self._check(self.lib.bem_profile_read(self.h, ctypes.byref(ms), ctypes.byref(nf), ctypes.byref(nk),
                                              1 if reset else 0))
        return {"far_ms": ms.value, "far_launches": nf.value, "kernel_launches": nk.value}


def quadrature_table(which, n=6):
    lib = _lib.load()
    buf = (ctypes.c_double * 256)()
    m = ctypes.c_int()
    check(lib.bem_quadrature_table(which, n, buf, ctypes.byref(m)))
    cols = 3 if which == 0 else 2
    return np.array(buf[:m.value * cols]).reshape(m.value, cols)
