"""Python binding of libsbfwi (argument marshalling only).

Every call goes to the C ABI declared in ``include/sbfwi.h``; nothing here
computes any part of the method.  Floating-point arrays may be numpy arrays (host
memory, staged by the library) or CUDA torch tensors (device memory, used in
place on torch's current stream).  If the compiled library is missing the import
fails loudly: there is no CPU fallback.
"""

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsbfwi.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ESTATE, ESINGULAR, EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
MEM_HOST, MEM_DEVICE = 0, 1
RHO_GRID, RHO_NODAL = 0, 1
GRAD_KERNEL, GRAD_EXACT = 0, 1
GRAD_ACCUMULATE = 0x100
CKPT_AUTO = -1
ELEMENT_AUTO, ELEMENT_TENSOR, ELEMENT_FP64, ELEMENT_MIXED = 0, 1, 2, 3
SOLVE_AUTO, SOLVE_DATAFLOW, SOLVE_BARRIER, SOLVE_LEVELS = 0, 1, 2, 3
TERMS_VELOCITY, TERMS_FULL = 0, 1
SESSION_FORWARD, SESSION_ADJOINT = 0, 1
PHASES = ("setup", "element", "solve", "other")

_NAMES = {EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA", ETIMEOUT: "ETIMEOUT", ESTATE: "ESTATE",
          ESINGULAR: "ESINGULAR", EUNSUPPORTED: "EUNSUPPORTED"}


class SbfwiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing; build it with paper_2501_06748_gb300.build.build() "
                          "(the library has no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I64, I32, D, VP = ctypes.POINTER, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
    pd, pi64 = P(ctypes.c_double), P(ctypes.c_int64)
    lib.sbfwi_last_error.restype = ctypes.c_char_p
    lib.sbfwi_version.restype = ctypes.c_int
    lib.sbfwi_build_mesh.argtypes = [P(VP), pd, I64, pi64, pi64, I64, pd, I64, I32, I32, D]
    lib.sbfwi_mesh_info.argtypes = [VP, pi64]
    lib.sbfwi_build_mesh3d.argtypes = [P(VP), pd, ctypes.c_int64, pi64, pi64, ctypes.c_int64, pd, ctypes.c_int64,
                                       I32, I32, ctypes.c_double]
    lib.sbfwi_build_mesh3d.restype = ctypes.c_int
    lib.sbfwi_set_model3d.argtypes = [P(VP), VP, ctypes.c_double, VP, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, VP]
    lib.sbfwi_set_model3d.restype = ctypes.c_int
    lib.sbfwi_destroy_mesh.argtypes = [VP]
    lib.sbfwi_destroy_mesh.restype = None
    lib.sbfwi_set_model.argtypes = [P(VP), VP, D, VP, ctypes.c_int, I64, I64, D, D, D, D, D, ctypes.c_int, VP]
    lib.sbfwi_set_model_lfe.argtypes = lib.sbfwi_set_model.argtypes
    lib.sbfwi_set_model_lfe.restype = ctypes.c_int
    lib.sbfwi_destroy_model.argtypes = [VP]
    lib.sbfwi_destroy_model.restype = None
    lib.sbfwi_forward.argtypes = [VP, I32, pi64, VP, I32, pi64, I64, VP, P(VP), I64, ctypes.c_int, VP]
    lib.sbfwi_misfit.argtypes = [VP, VP, I64, D, pd, VP, ctypes.c_int, VP]
    lib.sbfwi_adjoint_gradient.argtypes = [VP, VP, VP, ctypes.c_int, VP, ctypes.c_int, VP]
    lib.sbfwi_destroy_fwdstate.argtypes = [VP]
    lib.sbfwi_destroy_fwdstate.restype = None
    lib.sbfwi_misfit_noalloc.argtypes = [VP, VP, I64, D, VP, VP, VP]
    lib.sbfwi_misfit_noalloc.restype = ctypes.c_int
    lib.sbfwi_profile_enable.argtypes = [ctypes.c_int]
    lib.sbfwi_profile_read.argtypes = [pd, pi64, pi64, ctypes.c_int]
    lib.sbfwi_profile_solve_levels.argtypes = [pd, I32, P(I32), pi64, ctypes.c_int]
    lib.sbfwi_profile_solve_levels.restype = ctypes.c_int
    lib.sbfwi_profile_solve_flow.argtypes = [pd, I32, P(I32), pi64, ctypes.c_int]
    lib.sbfwi_profile_solve_flow.restype = ctypes.c_int
    lib.sbfwi_release_cache.argtypes = []
    lib.sbfwi_release_cache.restype = ctypes.c_int
    lib.sbfwi_lfe_element_matrices.argtypes = [pd, pd, pd, pd, I32, pd, pd]
    lib.sbfwi_lfe_element_matrices.restype = ctypes.c_int
    lib.sbfwi_set_kernel_terms.argtypes = [VP, ctypes.c_int]
    lib.sbfwi_set_kernel_terms.restype = ctypes.c_int
    lib.sbfwi_set_gradient_mode.argtypes = [VP, ctypes.c_int]
    lib.sbfwi_set_gradient_mode.restype = ctypes.c_int
    lib.sbfwi_set_schedule.argtypes = [VP, ctypes.c_int, ctypes.c_int]
    lib.sbfwi_set_schedule.restype = ctypes.c_int
    lib.sbfwi_session_create.argtypes = [P(VP), VP, I32, I32, I32, pi64, I32, VP]
    lib.sbfwi_session_admit.argtypes = [VP, I32, I64, VP, I64, VP, ctypes.c_int]
    lib.sbfwi_session_step.argtypes = [VP, P(I32)]
    lib.sbfwi_session_collect.argtypes = [VP, I32, VP, ctypes.c_int]
    lib.sbfwi_session_info.argtypes = [VP, pi64]
    lib.sbfwi_session_destroy.argtypes = [VP]
    lib.sbfwi_session_destroy.restype = None
    for name in ("sbfwi_session_create", "sbfwi_session_admit", "sbfwi_session_step", "sbfwi_session_collect",
                 "sbfwi_session_info"):
        getattr(lib, name).restype = ctypes.c_int
    lib.sbfwi_selftest_barrier.argtypes = [I32, I32, I64, I32, VP]
    lib.sbfwi_selftest_barrier.restype = ctypes.c_int
    for name in ("sbfwi_build_mesh", "sbfwi_mesh_info", "sbfwi_set_model", "sbfwi_forward", "sbfwi_misfit",
                 "sbfwi_adjoint_gradient", "sbfwi_profile_enable", "sbfwi_profile_read"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


_lib = _load()


def _check(code):
    if code != OK:
        raise SbfwiError(code, _lib.sbfwi_last_error().decode(errors="replace"))


def version() -> int:
    return _lib.sbfwi_version()


def profile_enable(on: bool = True) -> None:
    """Record CUDA-event timings of the library's kernel phases on their streams."""
    _check(_lib.sbfwi_profile_enable(1 if on else 0))


def profile_read(reset: bool = False) -> dict:
    """Per phase (setup, element, solve, other): device ms, timed intervals, kernel launches."""
    ms = np.zeros(4)
    iv = np.zeros(4, dtype=np.int64)
    la = np.zeros(4, dtype=np.int64)
    _check(_lib.sbfwi_profile_read(_dptr(ms), _iptr(iv), _iptr(la), 1 if reset else 0))
    return {ph: {"ms": float(ms[k]), "intervals": int(iv[k]), "launches": int(la[k])} for k, ph in enumerate(PHASES)}


def profile_solve_levels(reset: bool = False):
    """Per-phase timing (us) of the one-launch global solve while profiling was on
    (phases: forward levels leaves -> root, then backward levels root -> leaves).
    Returns (dict with 'wall' [2L] mean per solve seen by block 0, 'busy_max' [2L]
    longest time one block spent in a phase's tasks, 'busy_sum' [2L] mean per solve
    summed over blocks), solves recorded)."""
    cap = 256
    us = np.zeros(cap)
    n = ctypes.c_int32(0)
    steps = ctypes.c_int64(0)
    _check(_lib.sbfwi_profile_solve_levels(_dptr(us), cap, ctypes.byref(n), ctypes.byref(steps), 1 if reset else 0))
    k = n.value // 3
    return {"wall": us[:k].copy(), "busy_max": us[k:2 * k].copy(), "busy_sum": us[2 * k:3 * k].copy()}, int(steps.value)


def profile_solve_flow(reset: bool = False):
    """Per-phase timing (us) of the dataflow global solve while profiling was on (phases:
    forward levels leaves -> root, then backward levels root -> leaves).  Returns (dict with
    'done' [2L] time from the launch's start to the phase's last item finishing, 'exec' [2L]
    mean item execution time after its inputs were ready, 'wait' [2L] mean time an item
    waited for its inputs, 'items' [2L] items per solve), solves recorded)."""
    cap = 512
    us = np.zeros(cap)
    n = ctypes.c_int32(0)
    steps = ctypes.c_int64(0)
    _check(_lib.sbfwi_profile_solve_flow(_dptr(us), cap, ctypes.byref(n), ctypes.byref(steps), 1 if reset else 0))
    k = n.value // 4
    return ({"done": us[:k].copy(), "exec": us[k:2 * k].copy(), "wait": us[2 * k:3 * k].copy(),
             "items": us[3 * k:4 * k].copy()}, int(steps.value))


def _is_torch_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and hasattr(x, "data_ptr") and bool(x.is_cuda)


def _stream_of(x):
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)


def _f64_host(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i64_host(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


class _Arr:
    """A float64 array argument: host numpy or device torch tensor."""

    def __init__(self, a, writable=False):
        if _is_torch_cuda(a):
            import torch
            if a.dtype != torch.float64 or not a.is_contiguous():
                raise ValueError("device arrays must be contiguous float64 CUDA tensors")
            self.mem, self.ptr, self.obj, self.stream = MEM_DEVICE, ctypes.c_void_p(a.data_ptr()), a, _stream_of(a)
        else:
            if writable:
                if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
                    raise ValueError("host output arrays must be C-contiguous float64 numpy arrays")
                h = a
            else:
                h = _f64_host(a)
            self.mem, self.ptr, self.obj, self.stream = MEM_HOST, ctypes.c_void_p(h.ctypes.data), h, ctypes.c_void_p(None)


def _same_mem(*args):
    mems = {a.mem for a in args if a is not None}
    if len(mems) > 1:
        raise ValueError("mixing host and device arrays in one call is not supported")
    return mems.pop() if mems else MEM_HOST


class Mesh:
    def __init__(self, node_xy, elem_ptr, line_nodes, centre_xy, p, n_r, xi0=1e-3):
        """2-D: node_xy [N][2], line elements [L][p+1]; 3-D: node_xy [N][3] and faces
        [F][(p+1)^2] (sbfwi_build_mesh3d), told apart by the coordinate count."""
        xy, ep, ln, ct = _f64_host(node_xy), _i64_host(elem_ptr), _i64_host(line_nodes), _f64_host(centre_xy)
        self.dim = int(xy.shape[1])
        if self.dim not in (2, 3) or ct.shape[1] != self.dim:
            raise ValueError("node and centre coordinates must both be 2-D or both 3-D")
        h = ctypes.c_void_p()
        build = _lib.sbfwi_build_mesh3d if self.dim == 3 else _lib.sbfwi_build_mesh
        _check(build(ctypes.byref(h), _dptr(xy), xy.shape[0], _iptr(ep), _iptr(ln), ln.shape[0],
                     _dptr(ct), ct.shape[0], int(p), int(n_r), float(xi0)))
        self._h = h
        info = np.zeros(8, dtype=np.int64)
        _check(_lib.sbfwi_mesh_info(h, _iptr(info)))
        (self.n_elem, self.n_nodes, self.n_b, self.n_r, self.n_nodal, self.n_int,
         self.tree_levels, self.factor_entries) = (int(v) for v in info)

    @classmethod
    def from_inputs(cls, mesh, n_r, xi0=1e-3):
        """From an ``sbfwi_inputs`` mesh object (2-D, or 3-D from ``sbfwi_inputs.mesh3d``)."""
        if getattr(mesh, "dim", 2) == 3:
            return cls(mesh.node_xyz, mesh.elem_ptr, mesh.face_nodes, mesh.centre_xyz, mesh.p, n_r, xi0)
        return cls(mesh.node_xy, mesh.elem_ptr, mesh.line_nodes, mesh.centre_xy, mesh.p, n_r, xi0)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.sbfwi_destroy_mesh(h)
            self._h = None


class Model:
    def __init__(self, mesh: Mesh, c, rho, dt, beta=0.25, gamma=0.5, rho_kind=RHO_GRID, lx=1.0, ly=1.0, lfe=False,
                 lz=1.0):
        """``lfe=True``: the paper's comparison method (low-frequency expansion) instead of
        the radial finite differences.  On a 3-D mesh a grid density is [gz][gy][gx] on
        [0,lx]x[0,ly]x[0,lz] (sbfwi_set_model3d)."""
        r = _Arr(rho)
        h = ctypes.c_void_p()
        dim = getattr(mesh, "dim", 2)
        if dim == 3:
            if lfe:
                raise ValueError("the comparison method is built for 2-D meshes only")
            gz, gy, gx = (r.obj.shape if rho_kind == RHO_GRID else (0, 0, 0))
            _check(_lib.sbfwi_set_model3d(ctypes.byref(h), mesh._h, float(c), r.ptr, int(rho_kind), int(gx), int(gy),
                                          int(gz), float(lx), float(ly), float(lz), float(dt), float(beta),
                                          float(gamma), r.mem, r.stream))
        else:
            gz = 1
            gy, gx = (r.obj.shape if rho_kind == RHO_GRID else (0, 0))
            setup = _lib.sbfwi_set_model_lfe if lfe else _lib.sbfwi_set_model
            _check(setup(ctypes.byref(h), mesh._h, float(c), r.ptr, int(rho_kind), int(gx), int(gy),
                         float(lx), float(ly), float(dt), float(beta), float(gamma), r.mem, r.stream))
        self._h = h
        self.mesh = mesh                 # keeps the mesh alive for the model's lifetime
        self.rho_kind, self.gx, self.gy, self.gz, self.dt, self.lfe = (rho_kind, int(gx), int(gy), int(gz), float(dt),
                                                                       bool(lfe))

    @property
    def grad_shape(self):
        """Shape of the gradient on the model's parameter layout."""
        if self.rho_kind != RHO_GRID:
            return (self.mesh.n_nodal,)
        return (self.gz, self.gy, self.gx) if getattr(self.mesh, "dim", 2) == 3 else (self.gy, self.gx)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.sbfwi_destroy_model(h)
            self._h = None


class Session:
    """Continuous batching on one model (sbfwi_session_*): ``slots`` shot columns advanced in
    windows of ``window`` steps; requests are admitted into free slots between windows and
    collected when finished.  Forward requests give traces [R][K] (and, with ``field``, the
    nodal velocities for a later adjoint request); adjoint requests give the gradient of one
    shot.  Runs on torch's current stream of ``device``."""

    def __init__(self, model: "Model", kind, slots, rec_nodes, window=32, device=None):
        import torch
        self.model, self.kind = model, int(kind)
        self.rec = _i64_host(rec_nodes)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self._stream = ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        h = ctypes.c_void_p()
        _check(_lib.sbfwi_session_create(ctypes.byref(h), model._h, self.kind, int(slots), int(self.rec.size),
                                         _iptr(self.rec), int(window), self._stream))
        self._h = h
        info = self.info()
        self.field_stride, self.slots, self.window = info["field_stride"], info["slots"], info["window"]
        self._keep = {}                  # per slot: the arrays the library reads or writes asynchronously

    def info(self):
        v = np.zeros(5, dtype=np.int64)
        _check(_lib.sbfwi_session_info(self._h, _iptr(v)))
        return {"field_stride": int(v[0]), "steps": int(v[1]), "slots": int(v[2]), "window": int(v[3]),
                "busy": int(v[4])}

    def admit(self, slot, values, src_node=0, field=None):
        """Forward: values = wavelet [K] at ``src_node``; adjoint: values = residual [R][K].
        ``field``: a CUDA float64 tensor [K][field_stride] (forward: filled; adjoint: read)."""
        v = _Arr(values)
        K = int(v.obj.shape[-1])
        fptr = None
        if field is not None:
            if not _is_torch_cuda(field):
                raise ValueError("field must be a CUDA tensor")
            if tuple(field.shape) != (K, self.field_stride) or not field.is_contiguous():
                raise ValueError(f"field must be a contiguous [{K}][{self.field_stride}] tensor")
            fptr = ctypes.c_void_p(field.data_ptr())
        _check(_lib.sbfwi_session_admit(self._h, int(slot), int(src_node), v.ptr, K, fptr, v.mem))
        self._keep[int(slot)] = (v, field, K)

    def step(self):
        """One window; returns the slots holding a finished request."""
        fin = np.zeros(self.slots, dtype=np.int32)
        _check(_lib.sbfwi_session_step(self._h, fin.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
        return [int(s) for s in np.nonzero(fin)[0]]

    def collect(self, slot):
        """The finished request's result as a CUDA tensor (traces [R][K] or the gradient)."""
        import torch
        _, _, K = self._keep.pop(int(slot))
        if self.kind == SESSION_FORWARD:
            out = torch.empty((self.rec.size, K), dtype=torch.float64, device=self.device)
        else:
            m = self.model
            shape = m.grad_shape
            out = torch.zeros(shape, dtype=torch.float64, device=self.device)
        _check(_lib.sbfwi_session_collect(self._h, int(slot), ctypes.c_void_p(out.data_ptr()), MEM_DEVICE))
        return out

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.sbfwi_session_destroy(h)
            self._h = None


class FwdState:
    def __init__(self, h, model, n_shots, n_rec, K):
        self._h, self.model, self.n_shots, self.n_rec, self.K = h, model, n_shots, n_rec, K

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.sbfwi_destroy_fwdstate(h)
            self._h = None


def forward(model: Model, src_nodes, wavelets, rec_nodes, keep=True, traces_out=None, ckpt_every=0):
    """Forward solve; returns (traces [B][R][K], FwdState or None).  With ``keep``,
    ``ckpt_every`` = 0 stores the velocities of every step for the adjoint, c > 0 keeps
    checkpoints every c steps (recomputed in the adjoint), CKPT_AUTO picks c."""
    src = _i64_host(src_nodes)
    rec = _i64_host(rec_nodes)
    w = _Arr(wavelets)
    B = int(src.shape[0])
    K = int(w.obj.shape[-1])
    if traces_out is None:
        if w.mem == MEM_DEVICE:
            import torch
            traces_out = torch.empty((B, rec.shape[0], K), dtype=torch.float64, device=w.obj.device)
        else:
            traces_out = np.zeros((B, rec.shape[0], K))
    t = _Arr(traces_out, writable=True)
    mem = _same_mem(w, t)
    h = ctypes.c_void_p()
    _check(_lib.sbfwi_forward(model._h, B, _iptr(src), w.ptr, int(rec.shape[0]), _iptr(rec), K, t.ptr,
                              ctypes.byref(h) if keep else None, int(ckpt_every), mem,
                              w.stream if mem == MEM_DEVICE else t.stream))
    st = FwdState(h, model, B, int(rec.shape[0]), K) if keep else None
    return traces_out, st


def misfit(traces, observed, dt, residual_out=None, want_residual=True):
    """E = 0.5 dt sum (observed - traces)^2 and the residual observed - traces."""
    t, o = _Arr(traces), _Arr(observed)
    n = int(np.prod(t.obj.shape))
    if int(np.prod(o.obj.shape)) != n:
        raise ValueError("observed and traces must have the same number of samples")
    if residual_out is not None and int(np.prod(residual_out.shape)) != n:
        raise ValueError("residual_out must have as many samples as traces")
    if want_residual and residual_out is None:
        if t.mem == MEM_DEVICE:
            import torch
            residual_out = torch.empty_like(t.obj)
        else:
            residual_out = np.zeros(t.obj.shape)
    r = _Arr(residual_out, writable=True) if residual_out is not None else None
    mem = _same_mem(t, o, r)
    E = ctypes.c_double()
    _check(_lib.sbfwi_misfit(t.ptr, o.ptr, n, float(dt), ctypes.byref(E), r.ptr if r else None, mem,
                             t.stream if mem == MEM_DEVICE else None))
    return E.value, residual_out


def adjoint_gradient(model: Model, state: FwdState, residual, mode=GRAD_KERNEL, grad_out=None, accumulate=False):
    """Time-reversed adjoint and velocity Frechet kernel (``mode=GRAD_KERNEL``) or the exact
    derivative of the discrete misfit (``mode=GRAD_EXACT``, forward state made in that
    gradient mode); returns the gradient on the model's parameter layout ([gy][gx] grid or
    [n_nodal]).  ``accumulate`` adds into ``grad_out``."""
    if accumulate:
        if grad_out is None:
            raise ValueError("accumulate needs grad_out")
        mode = int(mode) | GRAD_ACCUMULATE
    r = _Arr(residual)
    if grad_out is None:
        shape = model.grad_shape
        if r.mem == MEM_DEVICE:
            import torch
            grad_out = torch.zeros(shape, dtype=torch.float64, device=r.obj.device)
        else:
            grad_out = np.zeros(shape)
    g = _Arr(grad_out, writable=True)
    mem = _same_mem(r, g)
    _check(_lib.sbfwi_adjoint_gradient(model._h, state._h, r.ptr, int(mode), g.ptr, mem,
                                       r.stream if mem == MEM_DEVICE else None))
    return grad_out


def misfit_noalloc(traces, observed, dt, E_out, residual_out=None):
    """Misfit for callers that cannot let the library allocate device memory.

    All arguments are CUDA float64 tensors (E_out has one element); the call only
    enqueues work on torch's current stream and keeps its partial sums in a fixed
    array inside the library.  Calls that may overlap on the GPU must be ordered
    on one stream (they share that array).
    """
    arrs = [_Arr(traces), _Arr(observed), _Arr(E_out, writable=True)]
    if residual_out is not None:
        arrs.append(_Arr(residual_out, writable=True))
    if any(a.mem != MEM_DEVICE for a in arrs):
        raise ValueError("misfit_noalloc takes CUDA tensors only")
    n = int(np.prod(arrs[0].obj.shape))
    # the C entry point cannot see the lengths of device arrays: check them here
    if int(np.prod(arrs[1].obj.shape)) != n:
        raise ValueError("observed and traces must have the same number of samples")
    if residual_out is not None and int(np.prod(arrs[3].obj.shape)) != n:
        raise ValueError("residual_out must have as many samples as traces")
    if int(np.prod(arrs[2].obj.shape)) < 1:
        raise ValueError("E_out needs at least one element")
    _check(_lib.sbfwi_misfit_noalloc(arrs[0].ptr, arrs[1].ptr, n, float(dt), arrs[2].ptr,
                                     arrs[3].ptr if residual_out is not None else None, arrs[0].stream))
    return E_out, residual_out


def lfe_element_matrices(E0, E1, E2, M0):
    """(K, M) of the low-frequency expansion for one element's coefficient matrices (host)."""
    mats = [np.ascontiguousarray(x, dtype=np.float64) for x in (E0, E1, E2, M0)]
    nb = mats[0].shape[0]
    K, M = np.empty((nb, nb)), np.empty((nb, nb))
    _check(_lib.sbfwi_lfe_element_matrices(*(_dptr(x) for x in mats), nb, _dptr(K), _dptr(M)))
    return K, M


def set_kernel_terms(model: Model, terms: int = TERMS_VELOCITY) -> None:
    """Velocity term only (the paper's kernel) or the full Frechet kernel for later
    forward/adjoint pairs on the model."""
    _check(_lib.sbfwi_set_kernel_terms(model._h, int(terms)))


def set_gradient_mode(model: Model, mode: int = GRAD_KERNEL) -> None:
    """GRAD_KERNEL (the paper's velocity kernel) or GRAD_EXACT (the exact derivative of the
    discrete misfit) for the forward states of later forward passes on the model."""
    _check(_lib.sbfwi_set_gradient_mode(model._h, int(mode)))


def set_schedule(model: Model, element: int = ELEMENT_AUTO, solve: int = SOLVE_AUTO) -> None:
    """Element kernel and global-solve schedule of the model's later time loops."""
    _check(_lib.sbfwi_set_schedule(model._h, int(element), int(solve)))


def release_cache() -> None:
    """Free the cached forward-field store that destroyed forward states leave behind."""
    _check(_lib.sbfwi_release_cache())


def selftest_barrier(n_blocks, n_absent=0, budget_cycles=2_000_000, rounds=8, stream=None) -> int:
    """Run the library's bounded grid barrier with `n_absent` blocks that never arrive.
    Returns the status code (OK, or ETIMEOUT when the wait gave up) instead of raising
    on ETIMEOUT; other errors raise SbfwiError."""
    code = _lib.sbfwi_selftest_barrier(int(n_blocks), int(n_absent), int(budget_cycles), int(rounds),
                                       ctypes.c_void_p(stream))
    if code not in (OK, ETIMEOUT):
        _check(code)
    return code
