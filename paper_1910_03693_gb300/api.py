"""Python face of the C ABI: one FRContext per mesh, tensors in, tensors out.

Every method forwards to the CUDA library on the current PyTorch stream.
Floating-point precision follows the tensor dtype (float64 -> FR_F64,
float32 -> FR_F32).  State tensors are in the library's bucketed layout;
``pack``/``unpack`` convert from/to the canonical FP64 layout.
"""
import ctypes as C

import numpy as np
import torch

from . import _lib

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = _lib.load()
    return _LIB


class FRError(RuntimeError):
    def __init__(self, what, status):
        msg = lib().fr_last_error().decode(errors="replace")
        super().__init__(f"{what}: {_lib.STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(st, what):
    if st != 0:
        raise FRError(what, st)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _prec(t, bf16_operators=False):
    if t.dtype == torch.float64 and not bf16_operators:
        return _lib.FR_F64
    if t.dtype == torch.float32:
        return _lib.FR_BF16OP if bf16_operators else _lib.FR_F32
    raise TypeError(f"unsupported dtype {t.dtype}" + (" (bfloat16 operators need FP32 buffers)" if bf16_operators else ""))


def _low_prec(name):
    if name == "df":
        return _lib.FR_DF
    if name == "f32":
        return _lib.FR_F32
    raise ValueError(f"low-precision residual must be 'df' or 'f32', not {name!r}")


def _jv_prec(jv_dtype):
    """torch.float64 / torch.float32, or "bf16op" for FP32 products with bfloat16 operators."""
    if isinstance(jv_dtype, str):
        if jv_dtype == "bf16op":
            return _lib.FR_BF16OP
        raise ValueError(f"unknown product precision {jv_dtype!r}")
    return _lib.FR_F64 if jv_dtype == torch.float64 else _lib.FR_F32


def _dev(t, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    return t


class FRContext:
    """Mesh, physics and degree limits of one FR discretisation on the GPU.

    ``mesh`` needs the attributes nd, geom_order, nodes [E, (g+1)^nd, nd],
    nbr [E, 2nd], nbr_face [E, 2nd], orient [E, 2nd] and p [E] (numpy arrays),
    with the conventions of ``include/fr.h``.
    """

    def __init__(self, mesh, gamma=1.4, mu=0.0, Pr=0.72, q_inf=None, p_min=None, p_max=None, flux="rusanov"):
        p = np.ascontiguousarray(mesh.p, dtype=np.int8)
        p_min = int(p.min()) if p_min is None else int(p_min)
        p_max = int(p.max()) if p_max is None else int(p_max)
        self._arrays = dict(
            nodes=np.ascontiguousarray(mesh.nodes, dtype=np.float64),
            nbr=np.ascontiguousarray(mesh.nbr, dtype=np.int32),
            nbr_face=np.ascontiguousarray(mesh.nbr_face, dtype=np.int8),
            orient=np.ascontiguousarray(mesh.orient, dtype=np.int8),
            p=p)
        a = self._arrays
        md = _lib.MeshDesc(int(mesh.nd), int(len(p)), int(mesh.geom_order),
                           a["nodes"].ctypes.data_as(C.POINTER(C.c_double)),
                           a["nbr"].ctypes.data_as(C.POINTER(C.c_int32)),
                           a["nbr_face"].ctypes.data_as(C.POINTER(C.c_int8)),
                           a["orient"].ctypes.data_as(C.POINTER(C.c_int8)),
                           a["p"].ctypes.data_as(C.POINTER(C.c_int8)))
        qi = (C.c_double * 5)(*([0.0] * 5))
        if q_inf is not None:
            for k, v in enumerate(np.asarray(q_inf, dtype=np.float64).reshape(-1)[:5]):
                qi[k] = float(v)
        if flux not in _lib.FLUX:
            raise ValueError(f"common flux must be one of {sorted(_lib.FLUX)}, not {flux!r}")
        ph = _lib.Physics(float(gamma), float(mu), float(Pr), qi, _lib.FLUX[flux])
        lim = _lib.Limits(p_min, p_max)
        h = C.c_void_p()
        torch.cuda.init()
        _check(lib().fr_create(C.byref(md), C.byref(ph), C.byref(lim), C.byref(h)), "fr_create")
        self.h = h
        self.nd = int(mesh.nd)
        self.nv = self.nd + 2
        self.n_elem = len(p)
        self.refresh_layout()

    # ------------------------------------------------------------------ admin
    def refresh_layout(self):
        info = _lib.LayoutInfo()
        _check(lib().fr_layout(self.h, C.byref(info)), "fr_layout")
        self.n_dof = int(info.n_dof)
        self.n_dof_capacity = int(info.n_dof_capacity)
        self.bucket_count = list(info.bucket_count)
        self.bucket_offset = list(info.bucket_offset)
        self.affine = bool(info.affine)

    def p_map(self):
        out = np.zeros(self.n_elem, dtype=np.int8)
        _check(lib().fr_get_p(self.h, out.ctypes.data_as(C.POINTER(C.c_int8))), "fr_get_p")
        return out

    def close(self):
        if getattr(self, "h", None):
            lib().fr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty(self, dtype=torch.float64, capacity=False):
        n = self.n_dof_capacity if capacity else self.n_dof
        return torch.empty(n, dtype=dtype, device="cuda")

    # ------------------------------------------------------------ conversions
    def pack(self, canon, dtype=torch.float64, out=None):
        """Canonical FP64 vector (CUDA tensor, or a host tensor: page-locked or
        pageable, copied by the library) -> state layout in ``dtype``."""
        if not (isinstance(canon, torch.Tensor) and canon.is_contiguous()):
            raise ValueError("canon must be a contiguous tensor")
        assert canon.dtype == torch.float64 and canon.numel() == self.n_dof
        out = self.empty(dtype) if out is None else _dev(out, "out")
        _check(lib().fr_pack(self.h, _ptr(canon), _ptr(out), _prec(out), _stream()), "fr_pack")
        return out

    def unpack(self, q, out=None):
        """State layout -> canonical FP64 vector; ``out`` may be a CUDA tensor or
        a host tensor (filled once the current stream reaches the copy)."""
        q = _dev(q, "q")
        out = torch.empty(self.n_dof, dtype=torch.float64, device="cuda") if out is None else out
        if not (out.dtype == torch.float64 and out.is_contiguous() and out.numel() == self.n_dof):
            raise ValueError("out must be a contiguous FP64 tensor of n_dof values")
        _check(lib().fr_unpack(self.h, _ptr(q), _prec(q), _ptr(out), _stream()), "fr_unpack")
        return out

    # ---------------------------------------------------------------- operators
    def residual(self, q, out=None, bf16_operators=False, double_float=False):
        """R(q) in the precision of q; ``bf16_operators`` (FP32 q): the operator
        matrices rounded to bfloat16 (the BF16-operator trial);
        ``double_float`` (FP64 q): FP64 in and out, evaluated in double-float
        arithmetic (pairs of FP32 values, about 48 significant bits)."""
        q = _dev(q, "q")
        out = torch.empty_like(q) if out is None else _dev(out, "out")
        if double_float:
            if q.dtype != torch.float64:
                raise TypeError("double-float evaluation takes and returns FP64 buffers")
            prec = _lib.FR_DF
        else:
            prec = _prec(q, bf16_operators)
        _check(lib().fr_residual(self.h, _ptr(q), _ptr(out), prec, _stream()), "fr_residual")
        return out

    def jvp(self, q, v, out=None, mode="exact", eps=1e-6, bf16_operators=False):
        q, v = _dev(q, "q"), _dev(v, "v")
        out = torch.empty_like(q) if out is None else _dev(out, "out")
        m = _lib.FR_JV_EXACT if mode == "exact" else _lib.FR_JV_FD
        _check(lib().fr_jvp(self.h, _ptr(q), _ptr(v), _ptr(out), _prec(q, bf16_operators), m, float(eps),
                            _stream()), "fr_jvp")
        return out

    def vjp(self, q, w, out=None, bf16_operators=False):
        q, w = _dev(q, "q"), _dev(w, "w")
        out = torch.empty_like(q) if out is None else _dev(out, "out")
        _check(lib().fr_vjp(self.h, _ptr(q), _ptr(w), _ptr(out), _prec(q, bf16_operators), _stream()), "fr_vjp")
        return out


    # -------------------------------------------------------- launch tuning
    def autotune(self, q64):
        """Time the launch configurations on the FP64 state q64 and keep the fastest."""
        q64 = _dev(q64, "q64")
        _check(lib().fr_autotune(self.h, _ptr(q64), _stream()), "fr_autotune")
        return self.tuning()

    def tuning(self):
        """{"epb": 42 ints [prec][kernel][P], "multi_launch": bool, "graphs": bool, "diag_metrics": bool,
        "fused_jvp": bool, "df_arnoldi": bool, "arnoldi_runs": bool, "tma_faces": bool, "device_gmres": bool,
        "f32_basis": bool}"""
        tab = (C.c_int32 * 42)()
        fl = C.c_int32(0)
        _check(lib().fr_tuning_get(self.h, tab, C.byref(fl)), "fr_tuning_get")
        return {"epb": [int(x) for x in tab], "multi_launch": bool(fl.value & 1), "graphs": bool(fl.value & 2),
                "diag_metrics": bool(fl.value & 4), "fused_jvp": bool(fl.value & 8),
                "df_arnoldi": bool(fl.value & 16), "arnoldi_runs": bool(fl.value & 32),
                "tma_faces": bool(fl.value & 64), "device_gmres": bool(fl.value & 128),
                "f32_basis": bool(fl.value & 256)}

    def set_tuning(self, t):
        """Set what `tuning()` returns; a missing "epb" keeps the table, missing switches default to on."""
        tab = (C.c_int32 * 42)(*[int(x) for x in t["epb"]]) if "epb" in t else None
        flags = ((1 if t.get("multi_launch", True) else 0) | (2 if t.get("graphs", True) else 0) |
                 (4 if t.get("diag_metrics", True) else 0) | (8 if t.get("fused_jvp", True) else 0) |
                 (16 if t.get("df_arnoldi", False) else 0) | (32 if t.get("arnoldi_runs", True) else 0) |
                 (64 if t.get("tma_faces", True) else 0) | (128 if t.get("device_gmres", True) else 0) |
                 (256 if t.get("f32_basis", True) else 0))
        _check(lib().fr_tuning_set(self.h, tab, flags), "fr_tuning_set")

    # ---------------------------------------------------------- instrumentation
    def device_status(self, clear=True):
        """The context's device status word (bit 0: a bounded wait gave up)."""
        v = C.c_int32(0)
        _check(lib().fr_device_status(self.h, C.byref(v), 1 if clear else 0), "fr_device_status")
        return int(v.value)

    def timing(self, enable=True):
        _check(lib().fr_timing(self.h, 1 if enable else 0), "fr_timing")

    def timing_select(self, names=None):
        """Time only the kernels named (an iterable of timing names; None: all);
        the others are counted with 0 ms."""
        arg = None if not names else ",".join(names).encode()
        _check(lib().fr_timing_select(self.h, arg), "fr_timing_select")

    def timing_report(self):
        """{kernel name: (launches, total device ms, algorithmic bytes, algorithmic flops)} and
        the launch count."""
        buf = C.create_string_buffer(1 << 16)
        n = C.c_int64(0)
        _check(lib().fr_timing_report(self.h, buf, len(buf), C.byref(n)), "fr_timing_report")
        out = {}
        for line in buf.value.decode().splitlines():
            name, cnt, ms, nbytes, nflops = line.split()
            out[name] = (int(cnt), float(ms), float(nbytes), float(nflops))
        return out, int(n.value)

    # --------------------------------------------------------------- solvers
    def gmres(self, q64, b, sigma, mode="exact", jv_dtype=torch.float64, eps=1e-6, m=30, rtol=0.1,
              max_it=100, out=None, reorth=0, precond=False):
        """Solve (sigma I - dR/dq(q64)) x = b from x = 0 (FP64 Arnoldi).

        ``reorth``: 0 one classical Gram-Schmidt pass (the default of the paper's
        Krylov library), 1 a second pass when needed (DGKS), 2 always two.
        ``precond``: left element-Jacobi preconditioning with the blocks of the
        last ``precond_build`` (tolerance on the preconditioned residual)."""
        q64, b = _dev(q64, "q64"), _dev(b, "b")
        assert q64.dtype == torch.float64 and b.dtype == torch.float64
        x = torch.empty_like(b) if out is None else _dev(out, "out")
        op = _lib.ShiftedOp(float(sigma), q64.data_ptr(),
                            _lib.FR_JV_EXACT if mode == "exact" else _lib.FR_JV_FD,
                            _jv_prec(jv_dtype), float(eps), 1 if precond else 0)
        opts = _lib.GmresOpts(int(m), float(rtol), int(max_it), int(reorth))
        st = _lib.GmresStats()
        _check(lib().gmres_solve(self.h, C.byref(op), _ptr(b), _ptr(x), C.byref(opts), C.byref(st), _stream()),
               "gmres_solve")
        return x, dict(iterations=st.iterations, restarts=st.restarts, converged=bool(st.converged),
                       rel_res=st.rel_res)

    @staticmethod
    def _tableau(A, b=None):
        S = len(A)
        tab = _lib.Tableau()
        tab.s = S
        for i in range(S):
            for j in range(S):
                tab.A[i * S + j] = float(A[i][j])
        bb = A[-1] if b is None else b
        for i in range(S):
            tab.b[i] = float(bb[i])
        return tab

    @staticmethod
    def _newton_opts(tol, dtau_init, dtau_max, mode, jv_dtype, eps, m, rtol, max_it, max_newton, max_halvings,
                     reorth, low_above, precond=False, low_precision="df"):
        return _lib.NewtonOpts(float(tol), float(dtau_init), float(dtau_max), int(max_newton), int(max_halvings),
                               _lib.FR_JV_EXACT if mode == "exact" else _lib.FR_JV_FD,
                               _jv_prec(jv_dtype), float(eps),
                               _lib.GmresOpts(int(m), float(rtol), int(max_it), int(reorth)), float(low_above),
                               1 if precond else 0, _low_prec(low_precision))

    # ------------------------------------------------ element-Jacobi preconditioner
    def precond_build(self, q64, sigma):
        """Element-Jacobi blocks of sigma I - dR/dq(q64), inverted (Sec. 2.3)."""
        q64 = _dev(q64, "q64")
        assert q64.dtype == torch.float64
        _check(lib().fr_precond_build(self.h, _ptr(q64), float(sigma), _stream()), "fr_precond_build")

    def precond_apply(self, w, out=None):
        """z = M^-1 w with the last built blocks (FP64 state layout)."""
        w = _dev(w, "w")
        z = torch.empty_like(w) if out is None else _dev(out, "out")
        _check(lib().fr_precond_apply(self.h, _ptr(w), _ptr(z), _stream()), "fr_precond_apply")
        return z

    def filter(self, q, alpha=0.2, p_above=2):
        """Nodal polynomial filter in place on ``q`` (FP64 state layout)."""
        q = _dev(q, "q")
        assert q.dtype == torch.float64
        _check(lib().fr_filter(self.h, _ptr(q), float(alpha), int(p_above), _stream()), "fr_filter")
        return q

    def precond_release(self):
        _check(lib().fr_precond_release(self.h), "fr_precond_release")

    @staticmethod
    def _stage_dict(st):
        return dict(newton=st.newton_iterations, gmres=st.gmres_iterations, halvings=st.halvings,
                    converged=bool(st.converged), norm0=st.norm0, norm_final=st.norm_final,
                    low_evaluations=st.low_evaluations, f64_evaluations=st.f64_evaluations)

    def esdirk_step(self, A, dt, q, b=None, adapt=None, tol=1e-8, dtau_init=0.05, dtau_max=10.0, mode="exact",
                    jv_dtype=torch.float32, eps=1e-6, m=30, rtol=0.1, max_it=100, max_newton=200,
                    max_halvings=20, reorth=0, low_above=0.0, low_precision="df", precond=False):
        """One ESDIRK time step in place on ``q`` (FP64 state layout; n_dof_capacity
        values when adapting).  ``adapt``: None, or dict(nu_max, nu_min, p_min,
        p_max, var) to run the indicator and the rebucketing after the step.
        Returns the per-stage statistics (stages 2..s)."""
        q = _dev(q, "q")
        assert q.dtype == torch.float64
        tab = self._tableau(A, b)
        o = self._newton_opts(tol, dtau_init, dtau_max, mode, jv_dtype, eps, m, rtol, max_it, max_newton,
                              max_halvings, reorth, low_above, precond, low_precision)
        stats = (_lib.StageStats * (len(A) - 1))()
        ad = None
        var = 1
        if adapt is not None:
            if q.numel() < self.n_dof_capacity:
                raise ValueError("q must hold n_dof_capacity values when adapting")
            ad = _lib.AdaptOpts(float(adapt.get("nu_max", 0.1)), float(adapt.get("nu_min", 0.001)),
                                int(adapt["p_min"]), int(adapt["p_max"]))
            var = int(adapt.get("var", 1))
        rc = lib().esdirk_step(self.h, C.byref(tab), float(dt), _ptr(q), C.byref(o), stats,
                               C.byref(ad) if ad is not None else None, var, _stream())
        if rc not in (0, -4):
            raise FRError("esdirk_step", rc)
        if adapt is not None:
            self.refresh_layout()
        return [self._stage_dict(st) for st in stats]

    def esdirk_stage(self, A, stage, dt, qn, Rstages, qi, tol=1e-8, dtau_init=0.05, dtau_max=10.0,
                     mode="exact", jv_dtype=torch.float32, eps=1e-6, m=30, rtol=0.1, max_it=100,
                     max_newton=200, max_halvings=20, b=None, reorth=0, low_above=0.0, low_precision="df",
                     precond=False):
        """Solve ESDIRK stage ``stage`` (1-based, >= 2) in place in ``qi``.

        ``A`` is the s x s tableau (list of rows); ``Rstages[j]`` holds R(q^{j+1})
        for j < stage-1 and receives R(q^stage) in slot stage-1 when not None.
        ``low_above`` > 0 (exact mode): F from the residual in
        ``low_precision`` ("df" double-float, or "f32") while ||F||/||F0|| is
        above it, FP64 below; convergence is decided in FP64."""
        S = len(A)
        tab = _lib.Tableau()
        tab.s = S
        for i in range(S):
            for j in range(S):
                tab.A[i * S + j] = float(A[i][j])
        bb = A[-1] if b is None else b
        for i in range(S):
            tab.b[i] = float(bb[i])
        ptrs = (C.c_void_p * S)(*[(r.data_ptr() if r is not None else 0) for r in Rstages])
        o = self._newton_opts(tol, dtau_init, dtau_max, mode, jv_dtype, eps, m, rtol, max_it, max_newton,
                              max_halvings, reorth, low_above, precond, low_precision)
        st = _lib.StageStats()
        rc = lib().esdirk_stage(self.h, C.byref(tab), int(stage), float(dt), _ptr(qn), ptrs, _ptr(qi),
                                C.byref(o), C.byref(st), _stream())
        if rc not in (0, -4):
            raise FRError("esdirk_stage", rc)
        return dict(newton=st.newton_iterations, gmres=st.gmres_iterations, halvings=st.halvings,
                    converged=bool(st.converged), norm0=st.norm0, norm_final=st.norm_final,
                    low_evaluations=st.low_evaluations, f64_evaluations=st.f64_evaluations)


    # ------------------------------------------------------------ adaptation
    def indicator(self, q, var=1, eta=None, eta_max=None):
        """Spectral decay indicator per element (element id order) and its maximum."""
        q = _dev(q, "q")
        eta = torch.empty(self.n_elem, dtype=torch.float64, device="cuda") if eta is None else eta
        eta_max = torch.empty(1, dtype=torch.float64, device="cuda") if eta_max is None else eta_max
        _check(lib().spectral_decay_indicator(self.h, _ptr(q), _prec(q), int(var), _ptr(eta), _ptr(eta_max),
                                              _stream()), "spectral_decay_indicator")
        return eta, eta_max

    def rebucket(self, eta, eta_max, q, nu_max=0.1, nu_min=0.001, p_min=None, p_max=None, perm=None):
        """Adapt the degrees and reorder ``q`` (capacity-sized state buffer) in place.
        Returns the element id at each new bucket position when ``perm`` is given."""
        q = _dev(q, "q")
        if q.numel() < self.n_dof_capacity:
            raise ValueError("q must hold n_dof_capacity values")
        pmn = int(self._arrays["p"].min()) if p_min is None else int(p_min)
        pmx = int(self._arrays["p"].max()) if p_max is None else int(p_max)
        o = _lib.AdaptOpts(float(nu_max), float(nu_min), pmn, pmx)
        _check(lib().p_rebucket(self.h, _ptr(eta), _ptr(eta_max), C.byref(o), _ptr(q), _prec(q), _ptr(perm),
                                _stream()), "p_rebucket")
        self.refresh_layout()
        return perm


DFLOAT_OPS = {"add": 0, "sub": 1, "mul": 2, "fma": 3, "div": 4, "sqrt": 5}


def dfloat_eval(op, a, b=None, c=None):
    """One double-float operation of the FR_DF arithmetic, elementwise on FP64
    CUDA tensors: "add", "sub", "mul", "fma" (a * b + c), "div", "sqrt"."""
    a = _dev(a, "a")
    out = torch.empty_like(a)
    ptr = lambda t: _ptr(_dev(t, "operand")) if t is not None else None
    _check(lib().fr_dfloat_eval(DFLOAT_OPS[op], _ptr(a), ptr(b), ptr(c), _ptr(out), a.numel(), _stream()),
           "fr_dfloat_eval")
    return out


def fma_rate(dtype=torch.float64, iters=4096):
    """Measured FMA throughput of the current GPU in TFLOP/s (FP64 or FP32)."""
    out = C.c_double(0.0)
    prec = _lib.FR_F64 if dtype == torch.float64 else _lib.FR_F32
    _check(lib().fr_fma_rate(prec, int(iters), C.byref(out), _stream()), "fr_fma_rate")
    return out.value


def esdirk_tableau(order=3):
    """(A, b) of the library's ESDIRK2 / ESDIRK3 tableau."""
    t = _lib.Tableau()
    _check(lib().fr_esdirk_tableau(int(order), C.byref(t)), "fr_esdirk_tableau")
    s = t.s
    return [[t.A[i * s + j] for j in range(s)] for i in range(s)], [t.b[i] for i in range(s)]


class _Residual(torch.autograd.Function):
    """R(q) with backward = VJP and forward-mode = exact JVP, both on the GPU."""

    @staticmethod
    def forward(q, ctx_h):
        return ctx_h.residual(q.contiguous())

    @staticmethod
    def setup_context(ctx, inputs, output):
        q, ctx_h = inputs
        ctx.save_for_backward(q)
        ctx.fr = ctx_h
        ctx.q_fw = q

    @staticmethod
    def backward(ctx, g):
        (q,) = ctx.saved_tensors
        return ctx.fr.vjp(q.contiguous(), g.contiguous()), None

    @staticmethod
    def jvp(ctx, dq, _):
        return ctx.fr.jvp(ctx.q_fw.contiguous(), dq.contiguous())


def autograd_residual(fr: FRContext, q: torch.Tensor) -> torch.Tensor:
    """Differentiable R(q) (reverse mode through fr_vjp, forward mode through fr_jvp)."""
    return _Residual.apply(q, fr)
