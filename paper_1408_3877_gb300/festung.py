"""ctypes binding of the festung C ABI (include/festung.h).

Argument marshalling only: every computation runs in the CUDA library.  Host arrays
are numpy arrays; device arrays are torch CUDA tensors (torch provides device memory
and streams).  Importing this module does not need a GPU; creating a context does.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfestung.so")

OK, EINVAL, EMESH, ENOMEM, ECUDA, ENOCONV, ESTATE, EDATA = 0, -1, -2, -3, -4, -5, -6, -7
HOST, DEVICE = 0, 1
FP64, FP32, MIXED, DFLOAT, BF16TAB, MIXED64 = 0, 1, 2, 3, 4, 5
SOLVER_CG, SOLVER_BICGSTAB = 1, 2
BATCH_UNION, BATCH_CONCURRENT = 0, 1
BDR_INTERIOR, BDR_DIRICHLET, BDR_NEUMANN = 0, 1, 2

EXPORTS = [
    "festung_mesh_create", "festung_setup", "festung_sizes", "festung_quad_points",
    "festung_set_coeff", "festung_set_source", "festung_set_bc", "festung_set_state",
    "festung_get_state", "festung_apply", "festung_apply_noalloc", "festung_step", "festung_solve_stationary",
    "festung_l2_error", "festung_get_flux",
    "festung_element_order", "festung_precond_blocks", "festung_launch_count", "festung_set_stream",
    "festung_last_error", "festung_destroy",
    "festung_autotune", "festung_fma_peak", "festung_warmstart_features", "festung_set_guess", "festung_set_coarse",
    "festung_set_precond_reuse", "festung_set_persistent", "festung_test_barrier_timeout",
    "festung_mlp_create", "festung_mlp_sizes", "festung_mlp_set_stream", "festung_mlp_forward", "festung_mlp_grad",
    "festung_mlp_adam", "festung_mlp_get", "festung_mlp_set", "festung_mlp_last_error", "festung_mlp_destroy",
    "festung_batch_create", "festung_batch_set_stream", "festung_batch_set_mode", "festung_batch_step",
    "festung_batch_launch_count",
    "festung_batch_last_error", "festung_batch_destroy",
]


class StepOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("prec", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int), ("solver", ctypes.c_int)]


class StepInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("solver", ctypes.c_int), ("symmetric", ctypes.c_int), ("fp64_iterations", ctypes.c_int),
                ("initial_rel_residual", ctypes.c_double), ("coarse_iterations", ctypes.c_int),
                ("precond_built", ctypes.c_int)]


class FestungError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("festung error %d: %s" % (code, msg))
        self.code = code


_lib = None


def load(path=None):
    """Load libfestung.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError("libfestung.so not built: run __graft_entry__.build() (%s missing)" % p)
    lib = ctypes.CDLL(p)
    vp, i64, dbl, cint = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    lib.festung_mesh_create.argtypes = [vp, i64, vp, i64, vp, ctypes.POINTER(vp)]
    lib.festung_setup.argtypes = [vp, cint, cint, dbl]
    lib.festung_sizes.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(cint), ctypes.POINTER(cint),
                                  ctypes.POINTER(cint)]
    lib.festung_quad_points.argtypes = [vp, vp, vp]
    lib.festung_set_coeff.argtypes = [vp, vp, cint]
    lib.festung_set_source.argtypes = [vp, vp, cint]
    lib.festung_set_bc.argtypes = [vp, vp, vp, cint]
    lib.festung_set_state.argtypes = [vp, vp, cint, cint]
    lib.festung_get_state.argtypes = [vp, vp, cint]
    lib.festung_apply.argtypes = [vp, vp, vp, cint, dbl]
    lib.festung_apply_noalloc.argtypes = [vp, vp, vp, cint, dbl]
    lib.festung_step.argtypes = [vp, dbl, ctypes.POINTER(StepOpts), ctypes.POINTER(StepInfo)]
    lib.festung_l2_error.argtypes = [vp, vp, ctypes.POINTER(dbl)]
    lib.festung_get_flux.argtypes = [vp, vp, ctypes.c_int]
    lib.festung_solve_stationary.argtypes = [vp, ctypes.POINTER(StepOpts), ctypes.POINTER(StepInfo)]
    lib.festung_set_stream.argtypes = [vp, vp]
    lib.festung_launch_count.argtypes = [vp, ctypes.POINTER(i64)]
    lib.festung_element_order.argtypes = [vp, vp]
    lib.festung_precond_blocks.argtypes = [vp, dbl, vp, vp]
    lib.festung_last_error.argtypes = [vp]
    lib.festung_last_error.restype = ctypes.c_char_p
    lib.festung_destroy.argtypes = [vp]
    lib.festung_destroy.restype = None
    lib.festung_autotune.argtypes = [vp, ctypes.POINTER(cint)]
    lib.festung_fma_peak.argtypes = [cint, ctypes.POINTER(dbl)]
    lib.festung_warmstart_features.argtypes = [vp, dbl, vp, vp, ctypes.POINTER(dbl)]
    lib.festung_set_guess.argtypes = [vp, vp, cint]
    lib.festung_set_coarse.argtypes = [vp, cint]
    lib.festung_set_precond_reuse.argtypes = [vp, cint]
    lib.festung_set_persistent.argtypes = [vp, cint]
    lib.festung_test_barrier_timeout.argtypes = [vp, cint]
    lib.festung_mlp_create.argtypes = [cint, cint, ctypes.c_uint64, ctypes.POINTER(vp)]
    lib.festung_mlp_sizes.argtypes = [vp, ctypes.POINTER(cint), ctypes.POINTER(cint), ctypes.POINTER(cint)]
    lib.festung_mlp_set_stream.argtypes = [vp, vp]
    lib.festung_mlp_forward.argtypes = [vp, vp, vp, i64]
    lib.festung_mlp_grad.argtypes = [vp, vp, vp, vp, i64, ctypes.POINTER(dbl)]
    lib.festung_mlp_adam.argtypes = [vp, dbl]
    lib.festung_mlp_get.argtypes = [vp, vp, vp]
    lib.festung_mlp_set.argtypes = [vp, vp]
    lib.festung_mlp_last_error.argtypes = []
    lib.festung_mlp_last_error.restype = ctypes.c_char_p
    lib.festung_mlp_destroy.argtypes = [vp]
    lib.festung_mlp_destroy.restype = None
    lib.festung_batch_create.argtypes = [vp, cint, ctypes.POINTER(vp)]
    lib.festung_batch_set_stream.argtypes = [vp, vp]
    lib.festung_batch_set_mode.argtypes = [vp, cint, cint]
    lib.festung_batch_step.argtypes = [vp, dbl, ctypes.POINTER(StepOpts), vp]
    lib.festung_batch_launch_count.argtypes = [vp, ctypes.POINTER(i64)]
    lib.festung_batch_last_error.argtypes = [vp]
    lib.festung_batch_last_error.restype = ctypes.c_char_p
    lib.festung_batch_destroy.argtypes = [vp]
    lib.festung_batch_destroy.restype = None
    for name in EXPORTS:
        if name not in ("festung_last_error", "festung_destroy", "festung_batch_last_error",
                        "festung_batch_destroy", "festung_mlp_last_error", "festung_mlp_destroy"):
            getattr(lib, name).restype = cint
    if path is None:
        _lib = lib
    return lib


def _ptr(a, dtype):
    """(pointer, loc, keepalive) of a numpy array or a torch CUDA tensor."""
    if a is None:
        return None, HOST, None
    if hasattr(a, "is_cuda") and a.is_cuda:
        if not a.is_contiguous():
            raise ValueError("device tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), DEVICE, a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(ctypes.c_void_p), HOST, arr


class Solver:
    """One mesh and its LDG discretisation on the current CUDA device."""

    def __init__(self, coordV, V0T, bdr_type):
        self.lib = load()
        cV = np.ascontiguousarray(coordV, dtype=np.float64)
        T = np.ascontiguousarray(V0T, dtype=np.int32)
        b = np.ascontiguousarray(bdr_type, dtype=np.int8)
        h = ctypes.c_void_p()
        rc = self.lib.festung_mesh_create(cV.ctypes.data, cV.shape[0], T.ctypes.data, T.shape[0], b.ctypes.data,
                                          ctypes.byref(h))
        if rc != OK:
            raise FestungError(rc, self.lib.festung_last_error(None).decode())
        self.h = h
        self.K = T.shape[0]
        self.N = self.R2 = self.R1 = None

    def _check(self, rc):
        if rc != OK:
            raise FestungError(rc, self.lib.festung_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.festung_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def setup(self, p, quad_order=0, eta=1.0):
        self._check(self.lib.festung_setup(self.h, p, quad_order, eta))
        K, N, R2, R1 = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.festung_sizes(self.h, ctypes.byref(K), ctypes.byref(N), ctypes.byref(R2),
                                           ctypes.byref(R1)))
        self.p, self.N, self.R2, self.R1 = p, N.value, R2.value, R1.value
        return self

    def quad_points(self):
        xy = np.zeros((self.K, self.R2, 2))
        exy = np.zeros((self.K, 3, self.R1, 2))
        self._check(self.lib.festung_quad_points(self.h, xy.ctypes.data, exy.ctypes.data))
        return xy, exy

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream (or None for the legacy default stream)."""
        self._check(self.lib.festung_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream if stream else 0)))

    def set_coeff(self, d_samples):
        p, loc, keep = _ptr(d_samples, np.float64)
        self._check(self.lib.festung_set_coeff(self.h, p, loc))

    def set_source(self, f_samples):
        p, loc, keep = _ptr(f_samples, np.float64)
        self._check(self.lib.festung_set_source(self.h, p, loc))

    def set_bc(self, cD=None, gN=None):
        p1, l1, k1 = _ptr(cD, np.float64)
        p2, l2, k2 = _ptr(gN, np.float64)
        loc = l1 if cD is not None else l2
        if cD is not None and gN is not None and l1 != l2:
            raise ValueError("cD and gN must both be host or both be device arrays")
        self._check(self.lib.festung_set_bc(self.h, p1, p2, loc))

    def set_state(self, C, is_samples=False):
        p, loc, keep = _ptr(C, np.float64)
        self._check(self.lib.festung_set_state(self.h, p, 1 if is_samples else 0, loc))

    def get_state(self, out=None):
        if out is None:
            out = np.zeros((self.K, self.N))
        p, loc, keep = _ptr(out, np.float64)
        if loc == HOST and keep is not out:
            raise ValueError("host output must be a contiguous float64 array")
        self._check(self.lib.festung_get_state(self.h, p, loc))
        return out

    def apply(self, x, y, dt, prec=FP64):
        """y = S x on device tensors of shape (N, K) in the internal triangle order: FP64 tensors for
        prec FP64 or DFLOAT (double-float evaluation), FP32 tensors for FP32 or BF16TAB (tables
        rounded to BF16)."""
        self._check(self.lib.festung_apply(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                           prec, dt))

    def step(self, dt, tol=1e-10, prec=MIXED, max_iter=20000, inner_tol=1e-2, max_outer=50, solver=0):
        o = StepOpts(tol, max_iter, prec, inner_tol, max_outer, solver)
        info = StepInfo()
        self._check(self.lib.festung_step(self.h, dt, ctypes.byref(o), ctypes.byref(info)))
        return {"iterations": info.iterations, "outer": info.outer, "rel_residual": info.rel_residual,
                "solver": info.solver, "symmetric": info.symmetric, "fp64_iterations": info.fp64_iterations,
                "initial_rel_residual": info.initial_rel_residual, "coarse_iterations": info.coarse_iterations,
                "precond_built": info.precond_built}

    def element_order(self):
        """order[i] = caller's index of the triangle at position i of the device layout."""
        o = np.zeros(self.K, dtype=np.int64)
        self._check(self.lib.festung_element_order(self.h, o.ctypes.data))
        return o

    def precond_blocks(self, dt):
        """(blocks, inverse), each K x N x N in the caller's order: the diagonal blocks S_kk
        of the step operator as the preconditioner build computes them, and the BF16
        inverses the Krylov kernels apply."""
        blocks = np.zeros((self.K, self.N, self.N))
        inverse = np.zeros((self.K, self.N, self.N))
        self._check(self.lib.festung_precond_blocks(self.h, dt, blocks.ctypes.data, inverse.ctypes.data))
        return blocks, inverse

    def launch_count(self):
        n = ctypes.c_int64()
        self._check(self.lib.festung_launch_count(self.h, ctypes.byref(n)))
        return n.value

    def solve_stationary(self, tol=1e-10, prec=MIXED, max_iter=100000, inner_tol=1e-2, max_outer=50, solver=0):
        """The stationary problem of Sec. 3.9 with the current coefficient, source and boundary data."""
        o = StepOpts(tol, max_iter, prec, inner_tol, max_outer, solver)
        info = StepInfo()
        self._check(self.lib.festung_solve_stationary(self.h, ctypes.byref(o), ctypes.byref(info)))
        return {"iterations": info.iterations, "outer": info.outer, "rel_residual": info.rel_residual,
                "solver": info.solver, "symmetric": info.symmetric, "fp64_iterations": info.fp64_iterations,
                "initial_rel_residual": info.initial_rel_residual, "coarse_iterations": info.coarse_iterations,
                "precond_built": info.precond_built}

    def set_persistent(self, enable=True):
        """FP32 BiCGStab at p <= 1 as one persistent kernel (1) or the graph of four kernels
        per iteration (0) (festung_set_persistent)."""
        self._check(self.lib.festung_set_persistent(self.h, 1 if enable else 0))
        return self

    def set_precond_reuse(self, max_steps):
        """One block-Jacobi build serves up to max_steps steps (festung_set_precond_reuse)."""
        self._check(self.lib.festung_set_precond_reuse(self.h, int(max_steps)))
        return self

    def set_coarse(self, enable=True):
        """Start every FP32 sweep from a coarse (p = 1) correction (festung_set_coarse)."""
        self._check(self.lib.festung_set_coarse(self.h, 1 if enable else 0))
        return self

    def autotune(self):
        """Pick the tile size of the fused apply by timing; returns it."""
        t = ctypes.c_int()
        self._check(self.lib.festung_autotune(self.h, ctypes.byref(t)))
        return t.value

    def warmstart_features(self, dt, X, Wt=None):
        """Features of the learned warm start into the device tensor X (K x (3 + 4N), FP32,
        internal order), optionally the loss weights into Wt (K x N); returns the residual scale rs."""
        sc = ctypes.c_double()
        wp = ctypes.c_void_p(Wt.data_ptr()) if Wt is not None else None
        self._check(self.lib.festung_warmstart_features(self.h, dt, ctypes.c_void_p(X.data_ptr()), wp,
                                                        ctypes.byref(sc)))
        return sc.value

    def set_guess(self, delta):
        """The next step starts from C^n + delta (K x N, caller order; None clears it)."""
        p, loc, keep = _ptr(delta, np.float64)
        self._check(self.lib.festung_set_guess(self.h, p, loc))

    def get_flux(self):
        """Z^1, Z^2 (each K x N, caller order) of the flux unknown z_h = -grad c_h from the current state."""
        Z = np.empty((2, self.K, self.N))
        self._check(self.lib.festung_get_flux(self.h, Z.ctypes.data, HOST))
        return Z

    def l2_error(self, c_samples):
        s = np.ascontiguousarray(c_samples, dtype=np.float64)
        e = ctypes.c_double()
        self._check(self.lib.festung_l2_error(self.h, s.ctypes.data, ctypes.byref(e)))
        return e.value


def _info_dict(info):
    return {"iterations": info.iterations, "outer": info.outer, "rel_residual": info.rel_residual,
            "solver": info.solver, "symmetric": info.symmetric, "fp64_iterations": info.fp64_iterations,
            "initial_rel_residual": info.initial_rel_residual, "coarse_iterations": info.coarse_iterations,
                "precond_built": info.precond_built}


class Batch:
    """Independent problems (set-up Solver objects) stepped together (festung_batch_*)."""

    def __init__(self, solvers):
        self.lib = load()
        self.solvers = list(solvers)
        arr = (ctypes.c_void_p * len(self.solvers))(*[s.h.value for s in self.solvers])
        h = ctypes.c_void_p()
        rc = self.lib.festung_batch_create(arr, len(self.solvers), ctypes.byref(h))
        if rc:
            raise FestungError(rc, self.lib.festung_batch_last_error(None).decode())
        self.h = h

    def _check(self, rc):
        if rc:
            raise FestungError(rc, self.lib.festung_batch_last_error(self.h).decode())

    def set_stream(self, stream):
        """Run on a torch.cuda.Stream (or a raw cudaStream_t as int)."""
        raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self._check(self.lib.festung_batch_set_stream(self.h, ctypes.c_void_p(raw)))

    def set_mode(self, mode, workers=0):
        """BATCH_CONCURRENT (the default: each problem its own step, `workers` at a time;
        0: 16, or the host's thread count if lower) or BATCH_UNION (joined meshes per group)."""
        self._check(self.lib.festung_batch_set_mode(self.h, mode, workers))

    def step(self, dt, tol=1e-10, max_iter=20000, inner_tol=1e-2, max_outer=50, solver=0):
        o = StepOpts(tol, max_iter, MIXED, inner_tol, max_outer, solver)
        infos = (StepInfo * len(self.solvers))()
        rc = self.lib.festung_batch_step(self.h, dt, ctypes.byref(o), infos)
        if rc:
            err = FestungError(rc, self.lib.festung_batch_last_error(self.h).decode())
            err.infos = [_info_dict(i) for i in infos]  # what each problem's step reported
            raise err
        return [_info_dict(i) for i in infos]

    def launch_count(self):
        n = ctypes.c_int64()
        self._check(self.lib.festung_batch_launch_count(self.h, ctypes.byref(n)))
        return n.value

    def close(self):
        if self.h:
            self.lib.festung_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLP:
    """The warm-start network (festung_mlp_*): in -> 64 -> 64 -> out, BF16 weights."""

    def __init__(self, n_in, n_out, seed=0):
        self.lib = load()
        h = ctypes.c_void_p()
        rc = self.lib.festung_mlp_create(n_in, n_out, seed, ctypes.byref(h))
        if rc:
            raise FestungError(rc, self.lib.festung_mlp_last_error().decode())
        self.h = h
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self.lib.festung_mlp_sizes(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
        self.n_in, self.n_out, self.n_params = a.value, b.value, c.value

    def _check(self, rc):
        if rc:
            raise FestungError(rc, self.lib.festung_mlp_last_error().decode())

    def set_stream(self, stream):
        raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self._check(self.lib.festung_mlp_set_stream(self.h, ctypes.c_void_p(raw)))

    def forward(self, X, Y):
        self._check(self.lib.festung_mlp_forward(self.h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                                 X.shape[0]))

    def grad(self, X, T, Wt=None):
        loss = ctypes.c_double()
        wp = ctypes.c_void_p(Wt.data_ptr()) if Wt is not None else None
        self._check(self.lib.festung_mlp_grad(self.h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(T.data_ptr()),
                                              wp, X.shape[0], ctypes.byref(loss)))
        return loss.value

    def adam(self, lr):
        self._check(self.lib.festung_mlp_adam(self.h, lr))

    def get(self):
        p = np.empty(self.n_params, dtype=np.float32)
        g = np.empty(self.n_params, dtype=np.float32)
        self._check(self.lib.festung_mlp_get(self.h, p.ctypes.data, g.ctypes.data))
        return p, g

    def set(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        self._check(self.lib.festung_mlp_set(self.h, p.ctypes.data))

    def close(self):
        if getattr(self, "h", None):
            self.lib.festung_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fma_peak(prec=FP32):
    """Measured multiply-add throughput of the current device (TFLOP/s)."""
    lib = load()
    t = ctypes.c_double()
    rc = lib.festung_fma_peak(prec, ctypes.byref(t))
    if rc:
        raise FestungError(rc, "festung_fma_peak failed")
    return t.value
