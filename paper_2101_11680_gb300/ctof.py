"""Python binding of the ctof C ABI (``include/ctof.h``).

Argument marshalling only: every step of the computation runs inside
``libctof.so``.  PyTorch supplies device memory and streams; tensors are passed
by ``data_ptr()`` and streams by their ``cuda_stream`` handle.  There is no
CPU fallback: if the library is missing, ``load()`` raises.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libctof.so")

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
LINEAR, CIRCULAR = 0, 1
SOLVER_ADMM_TV, SOLVER_TIKHONOV, SOLVER_FISTA_L1, SOLVER_FISTA_L1_MUX = 0, 1, 2, 3
KEEP_W = 1
FP32, BF16, FP8E4M3 = 0, 1, 2


class Optics(ctypes.Structure):
    _fields_ = [("mua_mm", ctypes.c_double), ("musp_mm", ctypes.c_double), ("n", ctypes.c_double),
                ("z0_mm", ctypes.c_double), ("clamp_r", ctypes.c_int)]


class Emission(ctypes.Structure):
    _fields_ = [("mua_mm", ctypes.c_double), ("musp_mm", ctypes.c_double), ("tau_ps", ctypes.c_double)]


class VoxelAverage(ctypes.Structure):
    _fields_ = [("layers", ctypes.c_int), ("nodes", ctypes.c_int)]


class GridSpec(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("nt", ctypes.c_int),
                ("dx_mm", ctypes.c_double), ("dy_mm", ctypes.c_double), ("dz_mm", ctypes.c_double),
                ("z_first_mm", ctypes.c_double), ("dt_ps", ctypes.c_double), ("conv_mode", ctypes.c_int)]


class KernelInfo(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("n_freq", ctypes.c_int), ("n_class", ctypes.c_int), ("nt", ctypes.c_int),
                ("nz", ctypes.c_int), ("scale", ctypes.c_double), ("gram_max_diag", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t), ("admm_stages", ctypes.c_int)]


class SolverParams(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int), ("iters", ctypes.c_int), ("rho", ctypes.c_double),
                ("tv_beta", ctypes.c_double), ("beta_rel", ctypes.c_double), ("tik_lambda_rel", ctypes.c_double)]


class Report(ctypes.Structure):
    _fields_ = [("scale", ctypes.c_double), ("beta", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("iters_done", ctypes.c_int)]


class Timing(ctypes.Structure):
    _fields_ = [("contract_ms", ctypes.c_double), ("t_side_ms", ctypes.c_double), ("z_side_ms", ctypes.c_double),
                ("iterations_ms", ctypes.c_double), ("contract_launches", ctypes.c_int),
                ("graph_kernel_nodes", ctypes.c_int)]


class CtofError(RuntimeError):
    def __init__(self, status, where):
        lib = load()
        msg = lib.ctof_status_string(status).decode()
        detail = lib.ctof_last_error_message().decode()
        super().__init__(f"{where}: {msg} ({status}){': ' + detail if detail else ''}")
        self.status = status


_lib = None

_P = ctypes.c_void_p
_SIGNATURES = {
    "ctof_build_kernel": (ctypes.c_int, [ctypes.POINTER(Optics), ctypes.POINTER(GridSpec), ctypes.c_int, _P,
                                         ctypes.POINTER(_P)]),
    "ctof_build_kernel_fluorescence": (ctypes.c_int, [ctypes.POINTER(Optics), ctypes.POINTER(Emission),
                                                      ctypes.POINTER(GridSpec), ctypes.c_int, _P,
                                                      ctypes.POINTER(_P)]),
    "ctof_build_kernel_ex": (ctypes.c_int, [ctypes.POINTER(Optics), ctypes.POINTER(Emission),
                                            ctypes.POINTER(VoxelAverage), ctypes.POINTER(GridSpec), ctypes.c_int,
                                            _P, ctypes.POINTER(_P)]),
    "ctof_kernel_destroy": (None, [_P]),
    "ctof_kernel_get_info": (ctypes.c_int, [_P, ctypes.POINTER(KernelInfo)]),
    "ctof_kernel_get_w": (ctypes.c_int, [_P, _P]),
    "ctof_kernel_get_classes": (ctypes.c_int, [_P, _P]),
    "ctof_kernel_get_what": (ctypes.c_int, [_P, _P]),
    "ctof_forward": (ctypes.c_int, [_P, _P, _P, _P]),
    "ctof_adjoint": (ctypes.c_int, [_P, _P, _P, _P]),
    "ctof_forward_multiplexed": (ctypes.c_int, [_P, _P, _P, _P]),
    "ctof_contract_forward_batch": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P]),
    "ctof_contract_adjoint_batch": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P]),
    "ctof_adjoint_multiplexed": (ctypes.c_int, [_P, _P, _P, _P]),
    "ctof_reconstruct": (ctypes.c_int, [_P, _P, ctypes.POINTER(SolverParams), _P, ctypes.POINTER(Report), _P]),
    "ctof_reconstruct_host": (ctypes.c_int, [_P, _P, ctypes.POINTER(SolverParams), _P, ctypes.POINTER(Report),
                                             _P]),
    "ctof_forward_static": (ctypes.c_int, [_P, _P, _P, _P]),
    "ctof_reconstruct_batch_tikhonov": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int,
                                                       ctypes.c_double, _P, ctypes.POINTER(ctypes.c_double), _P]),
    "ctof_reconstruct_batch": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                              ctypes.POINTER(SolverParams), ctypes.POINTER(_P), _P]),
    "ctof_kernel_autotune": (ctypes.c_int, [_P, _P]),
    "ctof_learned_param_count": (ctypes.c_int, [ctypes.c_int]),
    "ctof_learned_create": (ctypes.c_int, [ctypes.c_int, _P, _P, ctypes.POINTER(_P)]),
    "ctof_learned_destroy": (None, [_P]),
    "ctof_learned_get_params": (ctypes.c_int, [_P, _P]),
    "ctof_learned_loss_grad": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P, ctypes.POINTER(ctypes.c_double), _P,
                                              _P]),
    "ctof_learned_train_step": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P, ctypes.c_double,
                                               ctypes.POINTER(ctypes.c_double), _P]),
    "ctof_learned_reconstruct": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P, _P]),
    "ctof_learned_reconstruct_checked": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P, _P, _P]),
    "ctof_kernel_get_tuning": (ctypes.c_int, [_P, _P]),
    "ctof_set_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "ctof_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_longlong]),
    "ctof_sync_status": (ctypes.c_int, [_P, _P]),
    "ctof_get_timing": (ctypes.c_int, [_P, ctypes.POINTER(Timing)]),
    "ctof_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ctof_last_error_message": (ctypes.c_char_p, []),
}


def load():
    """Load libctof.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2101_11680_gb300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(status, where):
    if status != OK:
        raise CtofError(status, where)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, shape, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


def make_optics(mua=0.01, musp=1.0, n=1.4, z0=0.0, clamp_r=True):
    return Optics(float(mua), float(musp), float(n), float(z0), int(bool(clamp_r)))


def make_emission(mua=0.005, musp=0.8, tau=0.0):
    """Emission-wavelength optics [1/mm] and fluorescence lifetime [ps] of the fluorescence mode."""
    return Emission(float(mua), float(musp), float(tau))


def make_grid(n, nz, nt, dx, dz, z_first, dt, dy=None, mode="linear"):
    return GridSpec(int(n), int(n), int(nz), int(nt), float(dx), float(dx if dy is None else dy), float(dz),
                    float(z_first), float(dt), LINEAR if mode == "linear" else CIRCULAR)


def admm_params(iters=100, rho=1.0, tv_beta=-1.0, beta_rel=1e-3):
    return SolverParams(SOLVER_ADMM_TV, int(iters), float(rho), float(tv_beta), float(beta_rel), 1e-3)


def tikhonov_params(lambda_rel=1e-3):
    return SolverParams(SOLVER_TIKHONOV, 1, 1.0, -1.0, 1e-3, float(lambda_rel))


def fista_params(iters=100, lam_rel=1e-2, lam=-1.0, multiplexed=False):
    """FISTA for the layer-weighted L1 problem (Eq. 10); lam < 0 selects lam_rel * max|A^T m| (normalised).

    multiplexed=True: the composite problem of Eq. 12 (measurement y = S m)."""
    return SolverParams(SOLVER_FISTA_L1_MUX if multiplexed else SOLVER_FISTA_L1, int(iters), 1.0, float(lam),
                        float(lam_rel), 1e-3)


class LearnedOptions(ctypes.Structure):
    _fields_ = [("x0_lambda_rel", ctypes.c_double), ("dc_steps", ctypes.c_int), ("dc_lambda_rel", ctypes.c_double)]


class Learned:
    """The unrolled proximal-gradient solver with a 3-D CNN prox (``ctof_learned``)."""

    def __init__(self, stages, params, x0_lambda_rel=0.0, dc_steps=0, dc_lambda_rel=0.0):
        import numpy as np
        lib = load()
        self._lib = lib
        self.stages = int(stages)
        self.x0_lambda_rel = float(x0_lambda_rel)
        self.options = LearnedOptions(float(x0_lambda_rel), int(dc_steps), float(dc_lambda_rel))
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != lib.ctof_learned_param_count(self.stages):
            raise ValueError("parameter count mismatch")
        h = ctypes.c_void_p()
        _check(lib.ctof_learned_create(self.stages, p.ctypes.data_as(ctypes.c_void_p), ctypes.byref(self.options),
                                       ctypes.byref(h)),
               "ctof_learned_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.ctof_learned_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        import numpy as np
        out = np.empty(self._lib.ctof_learned_param_count(self.stages), dtype=np.float32)
        _check(self._lib.ctof_learned_get_params(self._h, out.ctypes.data_as(ctypes.c_void_p)),
               "ctof_learned_get_params")
        return out

    def loss_grad(self, kernel, m, mu, stream=None):
        import numpy as np
        b = int(m.shape[0])
        grad = np.empty(self._lib.ctof_learned_param_count(self.stages), dtype=np.float32)
        loss = ctypes.c_double()
        _check(self._lib.ctof_learned_loss_grad(
            self._h, kernel._h, b, _dev_ptr(m, (b,) + kernel._meas_shape(), "m"),
            _dev_ptr(mu, (b,) + kernel._vol_shape(), "mu"), ctypes.byref(loss),
            grad.ctypes.data_as(ctypes.c_void_p), _stream_handle(stream)), "ctof_learned_loss_grad")
        return loss.value, grad

    def train_step(self, kernel, m, mu, lr, want_loss=False, stream=None):
        b = int(m.shape[0])
        loss = ctypes.c_double()
        _check(self._lib.ctof_learned_train_step(
            self._h, kernel._h, b, _dev_ptr(m, (b,) + kernel._meas_shape(), "m"),
            _dev_ptr(mu, (b,) + kernel._vol_shape(), "mu"), float(lr),
            ctypes.byref(loss) if want_loss else None, _stream_handle(stream)), "ctof_learned_train_step")
        return loss.value if want_loss else None

    def reconstruct(self, kernel, m, out=None, stream=None):
        import torch
        b = int(m.shape[0])
        if out is None:
            out = torch.empty((b,) + kernel._vol_shape(), device=m.device, dtype=torch.float32)
        _check(self._lib.ctof_learned_reconstruct(
            self._h, kernel._h, b, _dev_ptr(m, (b,) + kernel._meas_shape(), "m"),
            _dev_ptr(out, (b,) + kernel._vol_shape(), "out"), _stream_handle(stream)), "ctof_learned_reconstruct")
        return out

    def reconstruct_checked(self, kernel, m, out=None, res=None, stream=None):
        """Inference plus each member's relative data residual ||A mu - m|| / ||m||
        (float64 CUDA tensor [batch]); returns (out, res)."""
        import torch
        b = int(m.shape[0])
        if out is None:
            out = torch.empty((b,) + kernel._vol_shape(), device=m.device, dtype=torch.float32)
        if res is None:
            res = torch.empty(b, device=m.device, dtype=torch.float64)
        if (not isinstance(res, torch.Tensor) or not res.is_cuda or res.dtype != torch.float64
                or not res.is_contiguous() or tuple(res.shape) != (b,)):
            raise TypeError("res must be a contiguous float64 CUDA tensor of shape (batch,)")
        _check(self._lib.ctof_learned_reconstruct_checked(
            self._h, kernel._h, b, _dev_ptr(m, (b,) + kernel._meas_shape(), "m"),
            _dev_ptr(out, (b,) + kernel._vol_shape(), "out"), ctypes.c_void_p(res.data_ptr()),
            _stream_handle(stream)), "ctof_learned_reconstruct_checked")
        return out, res


def reconstruct_batch(kernels, ms, params, outs=None, stream=None):
    """ADMM for several problems (one Kernel each) in one captured multi-stream graph."""
    import torch
    lib = load()
    n = len(kernels)
    if outs is None:
        outs = [torch.empty(k._vol_shape(), device=m.device, dtype=torch.float32) for k, m in zip(kernels, ms)]
    hs = (ctypes.c_void_p * n)(*[k._h.value for k in kernels])
    mp = (ctypes.c_void_p * n)(*[_dev_ptr(m, k._meas_shape(), "m").value for k, m in zip(kernels, ms)])
    op = (ctypes.c_void_p * n)(*[_dev_ptr(o, k._vol_shape(), "out").value for k, o in zip(kernels, outs)])
    _check(lib.ctof_reconstruct_batch(n, hs, mp, ctypes.byref(params), op, _stream_handle(stream)),
           "ctof_reconstruct_batch")
    return outs


class Kernel:
    """A built sensitivity kernel (``ctof_kernel``) bound to the current CUDA device."""

    def __init__(self, optics, grid, keep_w=False, stream=None, emission=None, average=None):
        """emission: None for the absorption kernel, or an ``Emission`` (``make_emission``) for the
        fluorescence-mode kernel (``optics`` then holds the excitation-wavelength optics).
        average: None, or (layers, nodes) to average the first ``layers`` depth layers over the voxel
        with ``nodes`` Gauss-Legendre points per axis."""
        lib = load()
        self._lib = lib
        self.optics = optics
        self.grid = grid
        self.emission = emission
        h = ctypes.c_void_p()
        flags = KEEP_W if keep_w else 0
        self.average = average
        if average is not None:
            av = VoxelAverage(int(average[0]), int(average[1]))
            _check(lib.ctof_build_kernel_ex(ctypes.byref(optics), ctypes.byref(emission) if emission is not None else None,
                                            ctypes.byref(av), ctypes.byref(grid), flags, _stream_handle(stream),
                                            ctypes.byref(h)), "ctof_build_kernel_ex")
        elif emission is None:
            _check(lib.ctof_build_kernel(ctypes.byref(optics), ctypes.byref(grid), flags, _stream_handle(stream),
                                         ctypes.byref(h)), "ctof_build_kernel")
        else:
            _check(lib.ctof_build_kernel_fluorescence(ctypes.byref(optics), ctypes.byref(emission),
                                                      ctypes.byref(grid), flags, _stream_handle(stream),
                                                      ctypes.byref(h)), "ctof_build_kernel_fluorescence")
        self._h = h
        info = KernelInfo()
        _check(lib.ctof_kernel_get_info(h, ctypes.byref(info)), "ctof_kernel_get_info")
        self.info = info

    @property
    def n(self):
        return self.grid.nx

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.ctof_kernel_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- bounded device waits ----
    def set_wait_limit(self, polls):
        """Polls before a device-side wait of this handle's kernels gives up (0: at once)."""
        _check(self._lib.ctof_set_wait_limit(self._h, int(polls)), "ctof_set_wait_limit")

    def sync_status(self, stream=None):
        """Synchronise and read (and clear) the handle's sticky device status; raises on a timeout."""
        _check(self._lib.ctof_sync_status(self._h, _stream_handle(stream)), "ctof_sync_status")

    # ---- profiling ----
    def set_timing(self, enable):
        _check(self._lib.ctof_set_timing(self._h, 1 if enable else 0), "ctof_set_timing")

    def get_timing(self):
        t = Timing()
        st = self._lib.ctof_get_timing(self._h, ctypes.byref(t))
        if st not in (OK, EUNSUPPORTED):
            _check(st, "ctof_get_timing")
        return t

    def autotune(self, stream=None):
        _check(self._lib.ctof_kernel_autotune(self._h, _stream_handle(stream)), "ctof_kernel_autotune")
        return self.tuning()

    def tuning(self):
        out = (ctypes.c_int * 4)()
        self._lib.ctof_kernel_get_tuning(self._h, out)
        return list(out)

    # ---- parity accessors (synchronous) ----
    def get_w(self):
        import numpy as np
        q = self.grid.nx if self.grid.conv_mode == LINEAR else self.info.p // 2 + 1
        out = np.empty((self.grid.nt, self.grid.nz, q, q), dtype=np.float64)
        _check(self._lib.ctof_kernel_get_w(self._h, out.ctypes.data_as(ctypes.c_void_p)), "ctof_kernel_get_w")
        return out

    def get_classes(self):
        import numpy as np
        out = np.empty((self.info.n_class, 4), dtype=np.int32)
        _check(self._lib.ctof_kernel_get_classes(self._h, out.ctypes.data_as(ctypes.c_void_p)),
               "ctof_kernel_get_classes")
        return out

    def get_what(self):
        import numpy as np
        out = np.empty((self.info.n_class, self.grid.nt, self.grid.nz), dtype=np.float32)
        _check(self._lib.ctof_kernel_get_what(self._h, out.ctypes.data_as(ctypes.c_void_p)),
               "ctof_kernel_get_what")
        return out

    # ---- operators ----
    def _vol_shape(self):
        return (self.grid.nz, self.grid.ny, self.grid.nx)

    def _meas_shape(self):
        return (self.grid.nt, self.grid.ny, self.grid.nx)

    def forward(self, mu, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self._meas_shape(), device=mu.device, dtype=torch.float32)
        _check(self._lib.ctof_forward(self._h, _dev_ptr(mu, self._vol_shape(), "mu"),
                                      _dev_ptr(out, self._meas_shape(), "out"), _stream_handle(stream)),
               "ctof_forward")
        return out

    def forward_static(self, mu, out, stream=None):
        """Allocation-free forward operator (scratch in the library's fixed device array).

        For callers that may not allocate device memory at the call site (inside a
        stream capture, real-time loops, frameworks owning all allocations): the
        caller supplies `out`; nothing is allocated here or in the library.
        """
        _check(self._lib.ctof_forward_static(self._h, _dev_ptr(mu, self._vol_shape(), "mu"),
                                             _dev_ptr(out, self._meas_shape(), "out"), _stream_handle(stream)),
               "ctof_forward_static")
        return out

    def adjoint(self, m, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self._vol_shape(), device=m.device, dtype=torch.float32)
        _check(self._lib.ctof_adjoint(self._h, _dev_ptr(m, self._meas_shape(), "m"),
                                      _dev_ptr(out, self._vol_shape(), "out"), _stream_handle(stream)),
               "ctof_adjoint")
        return out

    def forward_multiplexed(self, mu, out=None, stream=None):
        """y = S A mu (Eq. 12: Hadamard multiplexing over 8 x 8 scan blocks)."""
        import torch
        if out is None:
            out = torch.empty(self._meas_shape(), device=mu.device, dtype=torch.float32)
        _check(self._lib.ctof_forward_multiplexed(self._h, _dev_ptr(mu, self._vol_shape(), "mu"),
                                                  _dev_ptr(out, self._meas_shape(), "out"), _stream_handle(stream)),
               "ctof_forward_multiplexed")
        return out

    def adjoint_multiplexed(self, y, out=None, stream=None):
        """A^T S^T y."""
        import torch
        if out is None:
            out = torch.empty(self._vol_shape(), device=y.device, dtype=torch.float32)
        _check(self._lib.ctof_adjoint_multiplexed(self._h, _dev_ptr(y, self._meas_shape(), "y"),
                                                  _dev_ptr(out, self._vol_shape(), "out"), _stream_handle(stream)),
               "ctof_adjoint_multiplexed")
        return out

    # ---- per-frequency contractions on spectra (batched) ----
    @property
    def ldt(self):
        return (self.info.nt + 7) // 8 * 8

    @property
    def ldz(self):
        return (self.info.nz + 7) // 8 * 8

    def contract_forward_batch(self, spec_z, out=None, stream=None):
        """[nvol][n_freq][ldz][2] float32 spectra -> [nvol][n_freq][ldt][2] (ctof_contract_forward_batch)."""
        import torch
        nvol = spec_z.shape[0]
        if out is None:
            out = torch.zeros((nvol, self.info.n_freq, self.ldt, 2), device=spec_z.device, dtype=torch.float32)
        _check(self._lib.ctof_contract_forward_batch(
            self._h, nvol, _dev_ptr(spec_z, (nvol, self.info.n_freq, self.ldz, 2), "spec_z"),
            _dev_ptr(out, (nvol, self.info.n_freq, self.ldt, 2), "out"), _stream_handle(stream)),
            "ctof_contract_forward_batch")
        return out

    def contract_adjoint_batch(self, spec_t, out=None, stream=None):
        """[nvol][n_freq][ldt][2] float32 spectra -> [nvol][n_freq][ldz][2] (ctof_contract_adjoint_batch)."""
        import torch
        nvol = spec_t.shape[0]
        if out is None:
            out = torch.zeros((nvol, self.info.n_freq, self.ldz, 2), device=spec_t.device, dtype=torch.float32)
        _check(self._lib.ctof_contract_adjoint_batch(
            self._h, nvol, _dev_ptr(spec_t, (nvol, self.info.n_freq, self.ldt, 2), "spec_t"),
            _dev_ptr(out, (nvol, self.info.n_freq, self.ldz, 2), "out"), _stream_handle(stream)),
            "ctof_contract_adjoint_batch")
        return out

    def reconstruct(self, m, params, out=None, report=False, stream=None):
        import torch
        if out is None:
            out = torch.empty(self._vol_shape(), device=m.device, dtype=torch.float32)
        rep = Report()
        _check(self._lib.ctof_reconstruct(self._h, _dev_ptr(m, self._meas_shape(), "m"), ctypes.byref(params),
                                          _dev_ptr(out, self._vol_shape(), "out"),
                                          ctypes.byref(rep) if report else None, _stream_handle(stream)),
               "ctof_reconstruct")
        return (out, rep) if report else out

    def reconstruct_batch_tikhonov(self, m, precision=BF16, refine=2, lambda_rel=1e-3, out=None, stream=None):
        """Tikhonov for a batch m [B][nt][n][n] (device); returns (mu [B][nz][n][n], lambda)."""
        import torch
        b = int(m.shape[0])
        if out is None:
            out = torch.empty((b,) + self._vol_shape(), device=m.device, dtype=torch.float32)
        lam = ctypes.c_double()
        _check(self._lib.ctof_reconstruct_batch_tikhonov(
            self._h, b, _dev_ptr(m, (b,) + self._meas_shape(), "m"), int(precision), int(refine),
            float(lambda_rel), _dev_ptr(out, (b,) + self._vol_shape(), "out"), ctypes.byref(lam),
            _stream_handle(stream)), "ctof_reconstruct_batch_tikhonov")
        return out, lam.value

    def reconstruct_host(self, m_host, params, out_host, report=False, stream=None):
        """Host-buffer variant: m_host / out_host are CPU float32 tensors (pinned for speed)."""
        import torch
        for t, shp, nm in ((m_host, self._meas_shape(), "m_host"), (out_host, self._vol_shape(), "out_host")):
            if t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or tuple(t.shape) != shp:
                raise TypeError(f"{nm} must be a contiguous float32 CPU tensor of shape {shp}")
        rep = Report()
        _check(self._lib.ctof_reconstruct_host(self._h, ctypes.c_void_p(m_host.data_ptr()), ctypes.byref(params),
                                               ctypes.c_void_p(out_host.data_ptr()),
                                               ctypes.byref(rep) if report else None, _stream_handle(stream)),
               "ctof_reconstruct_host")
        return (out_host, rep) if report else out_host
