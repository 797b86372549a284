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
        names = {f[0] for f in o._fields_}
        for k, v in kw.items():
            if k not in names:
                raise TypeError(f"unknown solve option {k!r}")
            setattr(o, k, v)
        r = _lib.bem_solve_report()
        rc = self.lib.bem_solve(self.h, ctypes.byref(o), ctypes.byref(r))
        if rc not in (0, -4):
            self._check(rc)
        return {"iterations": r.iterations, "refinements": r.refinements, "residual": r.residual,
                "seconds": r.seconds, "converged": rc == 0}

    def solve_basis(self, **kw):
        """Solve every piston of the transducer alone and keep the solutions
        for superposition (bem_solve_basis); solve options as for solve()."""
        o = _lib.bem_solve_opts()
        check(self.lib.bem_default_solve_opts(ctypes.byref(o)))
        names = {f[0] for f in o._fields_}
        for k, v in kw.items():
            if k not in names:
                raise TypeError(f"unknown solve option {k!r}")
            setattr(o, k, v)
        r = _lib.bem_solve_report()
        rc = self.lib.bem_solve_basis(self.h, ctypes.byref(o), ctypes.byref(r))
        if rc not in (0, _lib.ERR_NOT_CONVERGED):
            self._check(rc)
        return {"iterations": r.iterations, "refinements": r.refinements, "residual": r.residual,
                "seconds": r.seconds, "converged": rc == 0}

    def superpose(self, weights):
        """Solutions (n_exc, n_dofs) for piston weights (n_exc, n_elem) from the basis."""
        W = np.ascontiguousarray(np.atleast_2d(weights), dtype=np.complex128)
        U = np.empty((W.shape[0], self.n_dofs), dtype=np.complex128)
        self._check(self.lib.bem_superpose(self.h, W.ctypes.data, W.shape[0], U.ctypes.data, 0))
        return U

    def solution(self, rhs=0):
        """System-order solution of excitation rhs: per domain [gamma_N; gamma_D]."""
        u = np.empty(self.n_dofs, dtype=np.complex128)
        self._check(self.lib.bem_get_solution(self.h, int(rhs), u.ctypes.data, 0))
        return u

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

    # ---- memory
    def memory(self):
        """(bytes held on the device now, most held so far)."""
        u, p = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.bem_memory_info(self.h, ctypes.byref(u), ctypes.byref(p)))
        return u.value, p.value

    def estimate_solve_bytes(self, n_exc=1, **solve):
        o = _lib.bem_solve_opts()
        check(self.lib.bem_default_solve_opts(ctypes.byref(o)))
        for k, v in solve.items():
            setattr(o, k, v)
        b = ctypes.c_int64()
        self._check(self.lib.bem_estimate_solve_bytes(self.h, int(n_exc), ctypes.byref(o), ctypes.byref(b)))
        return b.value

    # ---- measurement
    def autotune(self, precision=FP32, timed=True):
        """Pick the far-field source-chunk length by timing (bem_autotune)."""
        ct = ctypes.c_int32()
        ms = ctypes.c_double()
        self._check(self.lib.bem_autotune(self.h, int(precision), ctypes.byref(ct),
                                          ctypes.byref(ms) if timed else None))
        return {"chunk_tiles": ct.value, "ms": ms.value if timed else None}

    def profile(self, enable=True):
        self._check(self.lib.bem_profile_enable(self.h, 1 if enable else 0))

    def profile_read(self, reset=True):
        ms = ctypes.c_double()
        nf = ctypes.c_int64()
        nk = ctypes.c_int64()
        self._check(self.lib.bem_profile_read(self.h, ctypes.byref(ms), ctypes.byref(nf), ctypes.byref(nk),
                                              1 if reset else 0))
        return {"far_ms": ms.value, "far_launches": nf.value, "kernel_launches": nk.value}


def peak_probe(which, iters, stream=None):
    """Measured arithmetic rate (bem_peak_probe): which 0 packed FP32 FMA
    (flops/s), 1 MUFU sine (ops/s), 2 FP64 FMA (flops/s)."""
    lib = _lib.load()
    r = ctypes.c_double()
    check(lib.bem_peak_probe(int(which), int(iters), ctypes.c_void_p(stream or 0), ctypes.byref(r)))
    return r.value


def quadrature_table(which, n=6):
    lib = _lib.load()
    buf = (ctypes.c_double * 256)()
    m = ctypes.c_int()
    check(lib.bem_quadrature_table(which, n, buf, ctypes.byref(m)))
    cols = 3 if which == 0 else 2
    return np.array(buf[:m.value * cols]).reshape(m.value, cols)


def apply_group(contexts, xs, ys=None):
    """y_i = A_hat_i x_i for several contexts in one far-field launch, replayed
    from a captured CUDA graph while the same contexts and tensors are used
    (bem_apply_group).  xs, ys: complex128 CUDA tensors, one per context."""
    import torch
    n = len(contexts)
    assert n == len(xs) and n > 0
    ys = [torch.empty_like(x) for x in xs] if ys is None else ys
    for c, x, y in zip(contexts, xs, ys):
        assert x.is_cuda and x.dtype == torch.complex128 and x.is_contiguous() and x.numel() == c.n_dofs
        assert y.is_cuda and y.dtype == torch.complex128 and y.is_contiguous() and y.numel() == c.n_dofs
    hs = (ctypes.c_void_p * n)(*[c.h.value for c in contexts])
    xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    yp = (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys])
    contexts[0]._check(contexts[0].lib.bem_apply_group(hs, n, xp, yp))
    return ys


class Server:
    """Request loop for planning solves (bem_server_*): scenes stay resident on
    the device, requests of piston excitations are queued, batched per scene
    and solved concurrently across scenes under one device-memory budget."""

    def __init__(self, device: int = 0, slots: int = 2, max_batch_rhs: int = 64, hbm_budget_bytes: int = 150 << 30,
                 join: int = 1, **solve):
        self.lib = _lib.load()
        o = _lib.bem_server_opts()
        check(self.lib.bem_server_default_opts(ctypes.byref(o)))
        o.slots, o.max_batch_rhs, o.hbm_budget_bytes = int(slots), int(max_batch_rhs), int(hbm_budget_bytes)
        o.join = int(join)
        names = {f[0] for f in o.solve._fields_}
        for k, v in solve.items():
            if k not in names:
                raise TypeError(f"unknown solve option {k!r}")
            setattr(o.solve, k, v)
        h = ctypes.c_void_p()
        rc = self.lib.bem_server_create(ctypes.byref(h), device, ctypes.byref(o))
        if rc:
            raise _lib.BemError(rc, "bem_server_create failed")
        self.h = h
        self.device = device
        self.scenes = {}

    def close(self):
        if getattr(self, "h", None):
            self.lib.bem_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_context(self, ctx: Context) -> int:
        """Hand a configured Context (meshes, materials, transducer) to the
        server, which owns it from then on."""
        i = ctypes.c_int32()
        rc = self.lib.bem_server_add_scene(self.h, ctx.h, ctypes.byref(i))
        if rc:
            raise _lib.BemError(rc, self.lib.bem_last_error(ctx.h).decode())
        ctx.h = None  # owned by the server now
        n, ne, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        check(self.lib.bem_server_scene_info(self.h, i, ctypes.byref(n), ctypes.byref(ne), ctypes.byref(b)))
        self.scenes[i.value] = (n.value, ne.value)
        return i.value

    def add_scene(self, scene, transducer=None, omega_rho0=None, **ctx_opts) -> int:
        """A synth scene with its transducer (scene.transducer by default)."""
        c = Context.from_scene(scene, self.device, stream=0, **ctx_opts)
        tr = transducer if transducer is not None else scene.transducer
        w = omega_rho0 if omega_rho0 is not None else 2 * np.pi * scene.freq * scene.rho0
        c.set_transducer(tr["centres"], tr["normals"], tr["radii"], w)
        return self.add_context(c)

    def estimate(self, scene_id: int, n_exc: int = 1) -> int:
        """Device bytes admission reserves for a solve of n_exc excitations."""
        b = ctypes.c_int64()
        check(self.lib.bem_server_estimate(self.h, int(scene_id), int(n_exc), ctypes.byref(b)))
        return b.value

    def submit(self, scene_id: int, weights) -> int:
        W = np.ascontiguousarray(np.atleast_2d(weights), dtype=np.complex128)
        assert W.shape[1] == self.scenes[scene_id][1], "weights: one per piston"
        hnd = ctypes.c_int64()
        check(self.lib.bem_server_submit(self.h, int(scene_id), W.ctypes.data, W.shape[0], ctypes.byref(hnd)))
        return hnd.value

    def poll(self, handle: int) -> int:
        st = ctypes.c_int32()
        check(self.lib.bem_server_poll(self.h, int(handle), ctypes.byref(st)))
        return st.value

    def wait(self, handle: int, timeout: float = -1.0) -> int:
        st = ctypes.c_int32()
        rc = self.lib.bem_server_wait(self.h, int(handle), float(timeout), ctypes.byref(st))
        if rc not in (0, _lib.ERR_TIMEOUT):
            check(rc)
        return st.value

    def result(self, handle: int, n_exc: int, scene_id: int, release: bool = True):
        """(U [n_exc, n_dofs], report dict); raises on a failed request."""
        n = self.scenes[scene_id][0]
        U = np.empty((n_exc, n), dtype=np.complex128)
        r = _lib.bem_solve_report()
        lat = ctypes.c_double()
        be = ctypes.c_int64()
        rc = self.lib.bem_server_result(self.h, int(handle), U.ctypes.data, ctypes.byref(r), ctypes.byref(lat),
                                        ctypes.byref(be), 0)
        msg = self.error(handle) if rc else ""
        if release:
            self.lib.bem_server_result(self.h, int(handle), None, None, None, None, 1)
        if rc:
            raise _lib.BemError(rc, msg or f"request {handle} failed")
        return U, {"iterations": r.iterations, "refinements": r.refinements, "residual": r.residual,
                   "seconds": r.seconds, "latency_ms": lat.value, "batch_exc": be.value}

    def error(self, handle: int) -> str:
        return self.lib.bem_server_error(self.h, int(handle)).decode()

    def stats(self) -> dict:
        st = _lib.bem_server_stats()
        check(self.lib.bem_server_get_stats(self.h, ctypes.byref(st)))
        return {f[0]: getattr(st, f[0]) for f in st._fields_}
