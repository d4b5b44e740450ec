"""ctypes binding of libfetipe.so (argument marshalling only; every computation runs in the
library's CUDA kernels).  Raises on import if the library has not been built: there is no
CPU fallback.

Names follow the C ABI of include/fetipe.h: ``create``, ``assemble``, ``factor``, ``step``,
``run``, ``get_lambda``, ``get_lambda_keys``, ``get_fields``, ``apply_F``,
``apply_precond``, ``apply_projection``, ``get_dof_map``, ``get_local_matrix``, and ``plan``
(fp_plan: sizes and multiplier keys from the library's host topology builder, no device).
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfetipe.so")
if not os.path.exists(LIB_PATH):
    raise ImportError("libfetipe.so not built: run paper_2509_06673_gb300/build.py "
                      "(or __graft_entry__.build()) first")
_lib = ctypes.CDLL(LIB_PATH)

FP_OK = 0
STATUS_NAMES = {0: "FP_OK", 1: "FP_ERR_INVALID", 2: "FP_ERR_OOM", 3: "FP_ERR_CUDA",
                4: "FP_ERR_NOT_CONVERGED", 5: "FP_ERR_BREAKDOWN", 6: "FP_ERR_TIMEOUT",
                7: "FP_ERR_STATE"}
globals().update({name: code for code, name in STATUS_NAMES.items()})
FP_SOURCE_MANUFACTURED, FP_SOURCE_POINT, FP_SOURCE_MANUFACTURED_T = 0, 1, 2
FP_PREC_FP64, FP_PREC_MIXED = 0, 1
FP_PRECOND_DIRICHLET, FP_PRECOND_LUMPED, FP_PRECOND_NONE, FP_PRECOND_AUTO = 0, 1, 2, 3

EXPORTED = ["fp_create", "fp_assemble", "fp_factor", "fp_step", "fp_run", "fp_get_sizes", "fp_plan",
            "fp_get_lambda", "fp_get_lambda_keys", "fp_get_fields", "fp_get_subdomain", "fp_set_initial",
            "fp_checkpoint", "fp_restore", "fp_apply_F",
            "fp_apply_precond", "fp_apply_projection", "fp_apply_projection_noalloc",
            "fp_get_dof_map",
            "fp_get_local_matrix", "fp_get_step_timing", "fp_set_option", "fp_set_profiling",
            "fp_get_kernel_stats", "fp_get_tuning", "fp_learned_record", "fp_learned_use", "fp_learned_train",
            "fp_learned_num_samples", "fp_mlp_init", "fp_mlp_set_params", "fp_mlp_get_params",
            "fp_mlp_forward", "fp_mlp_loss_grad", "fp_last_error", "fp_destroy"]
MLP_NPARAM = 8 * 256 + 256 + 256 * 256 + 256 + 256 + 1


class MeshDesc(ctypes.Structure):
    _fields_ = [("nsub_x", ctypes.c_int), ("nsub_y", ctypes.c_int),
                ("cells_x", ctypes.POINTER(ctypes.c_int)), ("cells_y", ctypes.POINTER(ctypes.c_int)),
                ("poro_rows", ctypes.c_int), ("order_k", ctypes.c_int)]


class Params(ctypes.Structure):
    _fields_ = [("lame_lambda", ctypes.c_double), ("mu", ctypes.c_double),
                ("alpha", ctypes.c_double), ("c0", ctypes.c_double),
                ("perm_k", ctypes.c_double), ("mu_f", ctypes.c_double), ("tau", ctypes.c_double),
                ("perm", ctypes.POINTER(ctypes.c_double)), ("source", ctypes.c_int),
                ("src_i", ctypes.c_int), ("src_j", ctypes.c_int), ("q_omega", ctypes.c_double),
                ("precision", ctypes.c_int), ("precond", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_it", ctypes.c_int)]


class Sizes(ctypes.Structure):
    _fields_ = [("nsub", ctypes.c_int), ("n_floating", ctypes.c_int), ("n_lambda", ctypes.c_int),
                ("n_lambda_p", ctypes.c_int), ("n_dofs", ctypes.c_longlong),
                ("n_unode_total", ctypes.c_longlong), ("n_pnode_total", ctypes.c_longlong),
                ("factor_bytes", ctypes.c_longlong), ("max_half_band", ctypes.c_int)]


class KernelStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("total_ms", ctypes.c_double),
                ("bytes_per_launch", ctypes.c_double), ("flops_per_launch", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("factor_nb", ctypes.c_int), ("solve_wpc", ctypes.c_int), ("solve_chunk", ctypes.c_int),
                ("solve_ctas_per_sm", ctypes.c_int), ("factor_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("candidates", ctypes.c_int),
                ("explicit_ms", ctypes.c_double), ("precond", ctypes.c_int),
                ("precond_rate", ctypes.c_double * 2), ("precond_ms_per_it", ctypes.c_double * 2),
                ("solve_mmax", ctypes.c_int), ("mrhs_nr", ctypes.c_int * 2), ("mrhs_mt", ctypes.c_int * 2),
                ("mrhs_esz", ctypes.c_int * 2), ("factor_tc_ms", ctypes.c_double * 2),
                ("mrhs_ms", ctypes.c_double * 2), ("mrhs_prec", ctypes.c_int * 2)]


class StepStats(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int), ("iterations", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("true_rel_residual", ctypes.c_double),
                ("lambda0_learned", ctypes.c_int), ("guess_res_prev", ctypes.c_double),
                ("guess_res_learned", ctypes.c_double), ("restarts", ctypes.c_int),
                ("stagnations", ctypes.c_int), ("h2d_bytes", ctypes.c_longlong),
                ("d2h_bytes", ctypes.c_longlong), ("kernel_launches", ctypes.c_longlong)]


_vp = ctypes.c_void_p
_lib.fp_create.argtypes = [ctypes.POINTER(MeshDesc), ctypes.POINTER(Params), _vp, ctypes.POINTER(_vp)]
for _n in ("fp_assemble", "fp_factor"):
    getattr(_lib, _n).argtypes = [_vp]
_lib.fp_step.argtypes = [_vp, ctypes.POINTER(StepStats)]
_lib.fp_run.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(StepStats)]
_lib.fp_get_sizes.argtypes = [_vp, ctypes.POINTER(Sizes)]
_lib.fp_plan.argtypes = [ctypes.POINTER(MeshDesc), ctypes.POINTER(Params), ctypes.POINTER(Sizes), _vp]
_lib.fp_get_lambda.argtypes = [_vp, _vp, ctypes.c_int]
_lib.fp_get_lambda_keys.argtypes = [_vp, _vp]
_lib.fp_get_fields.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_int]
_lib.fp_get_subdomain.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.c_int]
_lib.fp_checkpoint.argtypes = [_vp, ctypes.c_char_p]
_lib.fp_set_initial.argtypes = [_vp, _vp, _vp]
_lib.fp_restore.argtypes = [_vp, ctypes.c_char_p]
for _n in ("fp_apply_F", "fp_apply_precond", "fp_apply_projection"):
    getattr(_lib, _n).argtypes = [_vp, _vp, _vp, ctypes.c_int]
_lib.fp_apply_projection_noalloc.argtypes = [_vp, _vp, _vp]
_lib.fp_get_dof_map.argtypes = [_vp, ctypes.c_int, _vp, _vp, ctypes.POINTER(ctypes.c_int)]
_lib.fp_get_local_matrix.argtypes = [_vp, ctypes.c_int, _vp]
_lib.fp_get_step_timing.argtypes = [_vp, _vp]
_lib.fp_set_option.argtypes = [_vp, ctypes.c_char_p, ctypes.c_double]
_lib.fp_set_profiling.argtypes = [_vp, ctypes.c_int]
_lib.fp_get_kernel_stats.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(KernelStats)]
_lib.fp_get_tuning.argtypes = [_vp, ctypes.POINTER(Tuning)]
_lib.fp_learned_record.argtypes = [_vp, ctypes.c_int, ctypes.c_longlong, ctypes.c_int]
_lib.fp_learned_use.argtypes = [_vp, ctypes.c_int]
_lib.fp_learned_train.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_ulonglong,
                                  ctypes.POINTER(ctypes.c_double)]
_lib.fp_learned_num_samples.argtypes = [_vp, ctypes.POINTER(ctypes.c_longlong)]
_lib.fp_mlp_init.argtypes = [_vp, ctypes.c_ulonglong]
_lib.fp_mlp_set_params.argtypes = [_vp, _vp, ctypes.c_int]
_lib.fp_mlp_get_params.argtypes = [_vp, _vp, ctypes.c_int]
_lib.fp_mlp_forward.argtypes = [_vp, _vp, ctypes.c_int, _vp]
_lib.fp_mlp_loss_grad.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_double)]
_lib.fp_last_error.argtypes = [_vp]
_lib.fp_last_error.restype = ctypes.c_char_p
_lib.fp_destroy.argtypes = [_vp]
_lib.fp_destroy.restype = None


class FetipeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def _ptr(a):
    """Host numpy array or torch tensor -> (pointer, on_device)."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError(type(a))


def _describe(case, precision=None):
    """(fp_mesh_desc, fp_params, arrays that must outlive the call) for a workloads.Case."""
    cx = np.ascontiguousarray(case.cells_x, dtype=np.int32)
    cy = np.ascontiguousarray(case.cells_y, dtype=np.int32)
    keep = [cx, cy]
    mesh = MeshDesc(case.nsub_x, case.nsub_y, cx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                    cy.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), case.poro_rows, case.order_k)
    perm_ptr = None
    if case.perm is not None:
        perm = np.ascontiguousarray(np.concatenate([np.asarray(p, dtype=np.float64) for p in case.perm]))
        keep.append(perm)
        perm_ptr = perm.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    src = {"manufactured": FP_SOURCE_MANUFACTURED, "point": FP_SOURCE_POINT,
           "manufactured_t": FP_SOURCE_MANUFACTURED_T}[case.source]
    prec = precision or case.precision
    par = Params(case.lame_lambda, case.mu, case.alpha, case.c0, case.perm_k, case.mu_f, case.tau,
                 perm_ptr, src, int(case.src_node[0]), int(case.src_node[1]), float(case.q_omega),
                 FP_PREC_MIXED if prec == "mixed" else FP_PREC_FP64,
                 {"dirichlet": FP_PRECOND_DIRICHLET, "lumped": FP_PRECOND_LUMPED, "none": FP_PRECOND_NONE,
                  "auto": FP_PRECOND_AUTO}[case.precond],
                 case.tol, case.max_it)
    return mesh, par, keep


def plan(case, precision=None, keys=False):
    """fp_plan: the sizes of ``case`` (and, with keys=True, its multiplier keys as an
    (n_lambda, 6) int32 array) computed on the host, without a CUDA device."""
    mesh, par, keep = _describe(case, precision)
    s = Sizes()
    st = _lib.fp_plan(ctypes.byref(mesh), ctypes.byref(par), ctypes.byref(s), None)
    if st != FP_OK:
        raise FetipeError(st, _lib.fp_last_error(None).decode())
    if not keys:
        return s
    k = np.empty((s.n_lambda, 6), dtype=np.int32)
    st = _lib.fp_plan(ctypes.byref(mesh), ctypes.byref(par), ctypes.byref(s), k.ctypes.data)
    if st != FP_OK:
        raise FetipeError(st, _lib.fp_last_error(None).decode())
    return s, k


def _current_cuda_device():
    """The CUDA device current when a handle is created (the handle's device), if torch knows it."""
    try:
        import torch
        return torch.cuda.current_device() if torch.cuda.is_available() else None
    except Exception:
        return None


class Solver:
    """One fetipe handle.  ``case`` is a workloads.Case."""

    def __init__(self, case, stream=None, precision=None):
        self._h = _vp()
        mesh, par, self._keep = _describe(case, precision)
        st = _lib.fp_create(ctypes.byref(mesh), ctypes.byref(par), stream, ctypes.byref(self._h))
        if st != FP_OK:
            raise FetipeError(st, _lib.fp_last_error(None).decode())
        self.case = case
        self._device = _current_cuda_device()
        s = Sizes()
        self._check(_lib.fp_get_sizes(self._h, ctypes.byref(s)))
        self.sizes = s

    def _check(self, st):
        if st != FP_OK:
            raise FetipeError(st, _lib.fp_last_error(self._h).decode())

    def close(self):
        if self._h:
            _lib.fp_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # pipeline -------------------------------------------------------------------
    def assemble(self):
        self._check(_lib.fp_assemble(self._h))

    def factor(self):
        self._check(_lib.fp_factor(self._h))

    def step(self, allow_failure=False):
        st = StepStats()
        rc = _lib.fp_step(self._h, ctypes.byref(st))
        if not allow_failure:
            self._check(rc)
        return {"status": rc, "step": st.step, "iterations": st.iterations,
                "rel_residual": st.rel_residual, "true_rel_residual": st.true_rel_residual,
                "lambda0_learned": st.lambda0_learned, "guess_res_prev": st.guess_res_prev,
                "guess_res_learned": st.guess_res_learned, "restarts": st.restarts,
                "stagnations": st.stagnations, "h2d_bytes": st.h2d_bytes, "d2h_bytes": st.d2h_bytes,
                "kernel_launches": st.kernel_launches}

    def run(self, n_steps):
        st = StepStats()
        self._check(_lib.fp_run(self._h, n_steps, ctypes.byref(st)))
        return {"step": st.step, "iterations": st.iterations, "rel_residual": st.rel_residual,
                "true_rel_residual": st.true_rel_residual}

    # outputs --------------------------------------------------------------------
    def get_lambda(self, out=None):
        out = np.empty(self.sizes.n_lambda) if out is None else out
        p, dev = _ptr(out)
        self._check(_lib.fp_get_lambda(self._h, p, dev))
        return out

    def get_lambda_keys(self):
        k = np.empty((self.sizes.n_lambda, 6), dtype=np.int32)
        self._check(_lib.fp_get_lambda_keys(self._h, k.ctypes.data))
        return k

    def get_fields(self):
        s = self.sizes
        u = np.empty(2 * s.n_unode_total)
        xi = np.empty(s.n_pnode_total)
        eta = np.empty(s.n_pnode_total)
        p = np.empty(s.n_pnode_total)
        self._check(_lib.fp_get_fields(self._h, u.ctypes.data, xi.ctypes.data, eta.ctypes.data,
                                       p.ctypes.data, 0))
        return u, xi, eta, p

    def get_subdomain(self, s):
        """(u, xi, eta, p) of subdomain s, u as an (n_unode, 2) array (same as split_fields)."""
        c = self.case
        k = c.order_k
        if not 0 <= s < c.nsub:   # the library reports the bad index
            self._check(_lib.fp_get_subdomain(self._h, int(s), None, None, None, None, 0))
        nx, ny = c.cells_x[s % c.nsub_x], c.cells_y[s // c.nsub_x]
        u = np.empty(2 * (k * nx + 1) * (k * ny + 1))
        xi, eta, p = (np.empty((nx + 1) * (ny + 1)) for _ in range(3))
        self._check(_lib.fp_get_subdomain(self._h, int(s), u.ctypes.data, xi.ctypes.data, eta.ctypes.data,
                                          p.ctypes.data, 0))
        return u.reshape(-1, 2), xi, eta, p

    def set_initial(self, u0=None, p0=None):
        """Initial nodal fields in the layout of get_fields (None: zero)."""
        u = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64)
        p = None if p0 is None else np.ascontiguousarray(p0, dtype=np.float64)
        self._check(_lib.fp_set_initial(self._h, None if u is None else u.ctypes.data,
                                        None if p is None else p.ctypes.data))

    def checkpoint(self, path):
        self._check(_lib.fp_checkpoint(self._h, str(path).encode()))

    def restore(self, path):
        self._check(_lib.fp_restore(self._h, str(path).encode()))

    def _op(self, fn, v):
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.empty_like(v)
        self._check(fn(self._h, v.ctypes.data, out.ctypes.data, 0))
        return out

    def apply_F(self, v):
        return self._op(_lib.fp_apply_F, v)

    def apply_precond(self, v):
        return self._op(_lib.fp_apply_precond, v)

    def apply_projection(self, v):
        return self._op(_lib.fp_apply_projection, v)

    def apply_projection_noalloc(self, v, out):
        """fp_apply_projection_noalloc.  v, out: contiguous float64 CUDA tensors of n_lambda
        entries on the handle's device (out may be v).  torch's current stream is synchronised
        first, so that v is complete when the library's stream reads it."""
        import torch
        n = self.sizes.n_lambda
        for name, t in (("v", v), ("out", out)):
            if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda \
                    or not t.is_contiguous() or t.numel() != n:
                raise ValueError("%s must be a contiguous float64 CUDA tensor of %d entries" % (name, n))
        if v.device != out.device or (self._device is not None and v.device.index != self._device):
            raise ValueError("v and out must be on the handle's device (cuda:%s)" % self._device)
        torch.cuda.current_stream(v.device).synchronize()
        self._check(_lib.fp_apply_projection_noalloc(self._h, v.data_ptr(), out.data_ptr()))
        return out

    # learned initial guess -----------------------------------------------------
    def learned_record(self, on=True, max_samples=4_000_000, per_step=65536):
        self._check(_lib.fp_learned_record(self._h, 1 if on else 0, int(max_samples), int(per_step)))

    def learned_use(self, on=True):
        self._check(_lib.fp_learned_use(self._h, 1 if on else 0))

    def learned_train(self, epochs, batch=8192, lr=1e-3, seed=0):
        loss = ctypes.c_double()
        self._check(_lib.fp_learned_train(self._h, epochs, batch, lr, seed, ctypes.byref(loss)))
        return loss.value

    def learned_num_samples(self):
        n = ctypes.c_longlong()
        self._check(_lib.fp_learned_num_samples(self._h, ctypes.byref(n)))
        return n.value

    def mlp_init(self, seed):
        self._check(_lib.fp_mlp_init(self._h, seed))

    def mlp_set_params(self, theta):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        self._check(_lib.fp_mlp_set_params(self._h, t.ctypes.data, t.size))

    def mlp_get_params(self):
        t = np.empty(MLP_NPARAM, dtype=np.float32)
        self._check(_lib.fp_mlp_get_params(self._h, t.ctypes.data, t.size))
        return t

    def mlp_forward(self, x):
        x = np.ascontiguousarray(x, dtype=np.float32)
        out = np.empty(x.shape[0], dtype=np.float32)
        self._check(_lib.fp_mlp_forward(self._h, x.ctypes.data, x.shape[0], out.ctypes.data))
        return out

    def mlp_loss_grad(self, x, y):
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        g = np.empty(MLP_NPARAM, dtype=np.float32)
        loss = ctypes.c_double()
        self._check(_lib.fp_mlp_loss_grad(self._h, x.ctypes.data, y.ctypes.data, x.shape[0], g.ctypes.data,
                                          ctypes.byref(loss)))
        return loss.value, g

    def get_dof_map(self, s):
        n = ctypes.c_int()
        self._check(_lib.fp_get_dof_map(self._h, s, None, None, ctypes.byref(n)))
        f = np.empty(n.value, dtype=np.int32)
        nd = np.empty(n.value, dtype=np.int32)
        self._check(_lib.fp_get_dof_map(self._h, s, f.ctypes.data, nd.ctypes.data, ctypes.byref(n)))
        return f, nd

    def get_local_matrix(self, s):
        f, _ = self.get_dof_map(s)
        A = np.empty((f.size, f.size))
        self._check(_lib.fp_get_local_matrix(self._h, s, A.ctypes.data))
        return A

    def set_option(self, key, value):
        self._check(_lib.fp_set_option(self._h, key.encode(), float(value)))

    def set_profiling(self, on=True):
        self._check(_lib.fp_set_profiling(self._h, 1 if on else 0))

    def tuning(self):
        t = Tuning()
        self._check(_lib.fp_get_tuning(self._h, ctypes.byref(t)))
        out = {k: getattr(t, k) for k, _ in Tuning._fields_}
        for k in ("precond_rate", "precond_ms_per_it", "mrhs_nr", "mrhs_mt", "mrhs_esz", "factor_tc_ms", "mrhs_ms", "mrhs_prec"):
            out[k] = list(out[k])
        return out

    def kernel_stats(self, kind):
        s = KernelStats()
        self._check(_lib.fp_get_kernel_stats(self._h, kind, ctypes.byref(s)))
        return {"launches": s.launches, "total_ms": s.total_ms,
                "bytes_per_launch": s.bytes_per_launch, "flops_per_launch": s.flops_per_launch}

    def step_timing(self):
        t = np.zeros(4)
        self._check(_lib.fp_get_step_timing(self._h, t.ctypes.data))
        return t


def split_fields(case, u, xi, eta, p):
    """Per-subdomain views of the canonical field arrays (same layout as the C ABI)."""
    out = []
    ou = op = 0
    k = case.order_k
    for s in range(case.nsub):
        nx = case.cells_x[s % case.nsub_x]
        ny = case.cells_y[s // case.nsub_x]
        nun = (k * nx + 1) * (k * ny + 1)
        npn = (nx + 1) * (ny + 1)
        out.append((u[2 * ou: 2 * (ou + nun)].reshape(-1, 2), xi[op: op + npn], eta[op: op + npn],
                    p[op: op + npn]))
        ou += nun
        op += npn
    return out
