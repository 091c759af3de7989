"""Thin ctypes binding of libhelm.so (the C ABI in include/helm.h).

Argument marshalling only: every numerical step runs in the CUDA library.  Device memory and
streams come from PyTorch tensors.  Importing this module loads the library and raises if it is
missing (run `python -m paper_2607_16906_b300.build`); there is no CPU fallback.

Batch vectors are CUDA tensors of dtype complex64 (HELM_C64) or complex128 (HELM_C128), laid out
[system][rhs][Ny][Nx] flattened in system order, contiguous.
"""
from __future__ import annotations

import ctypes as ct
import functools
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhelm.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"libhelm.so not found at {LIB_PATH}; build it with `python -m paper_2607_16906_b300.build`")
_lib = ct.CDLL(LIB_PATH)

HELM_OK, HELM_ERR_INVALID_ARG, HELM_ERR_CUDA, HELM_ERR_OOM = 0, 1, 2, 3
HELM_NOT_CONVERGED, HELM_BREAKDOWN, HELM_NAN, HELM_TIMEOUT = 4, 5, 6, 7
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "NOT_CONVERGED", 5: "BREAKDOWN", 6: "NAN",
                7: "TIMEOUT"}
HELM_C64, HELM_C128 = 0, 1
HELM_MAX_M = 4096
HELM_MAX_COLUMNS = 65535
HELM_LAYER_DEC1B_FINAL = 17
HELM_FAULT_NONE, HELM_FAULT_STENCIL_TILE, HELM_FAULT_CONV_TILE, HELM_FAULT_ALLOC = 0, 1, 2, 3


class helm_grid(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int), ("h", ct.c_double)]


class helm_pml(ct.Structure):
    _fields_ = [("width", ct.c_int), ("sigma_max", ct.c_double)]


class helm_solve_opts(ct.Structure):
    _fields_ = [("m", ct.c_int), ("max_restarts", ct.c_int), ("max_outer", ct.c_int), ("tol", ct.c_double),
                ("inner_tol", ct.c_double), ("mixed", ct.c_int), ("orth", ct.c_int)]


class helm_solve_info(ct.Structure):
    _fields_ = [("iters", ct.c_int), ("restarts", ct.c_int), ("outer", ct.c_int), ("relres_true", ct.c_double),
                ("relres_est", ct.c_double), ("status", ct.c_int)]


_P = ct.c_void_p
_SIGS = {
    "helm_create": (ct.c_int, [ct.POINTER(_P), ct.c_int, ct.POINTER(helm_grid), ct.POINTER(helm_pml),
                               ct.POINTER(ct.c_double), _P, ct.c_int, _P]),
    "helm_destroy": (ct.c_int, [_P]),
    "helm_set_velocity": (ct.c_int, [_P, _P, ct.c_int, _P]),
    "helm_points": (ct.c_int64, [_P]),
    "helm_num_systems": (ct.c_int, [_P]),
    "helm_apply": (ct.c_int, [_P, _P, _P, ct.c_int, ct.c_int, _P]),
    "helm_apply_adjoint": (ct.c_int, [_P, _P, _P, ct.c_int, ct.c_int, _P]),
    "helm_apply_fourier": (ct.c_int, [_P, _P, _P, ct.c_int, ct.c_int, _P]),
    "helm_relres": (ct.c_int, [_P, _P, _P, ct.c_int, ct.POINTER(ct.c_double), _P]),
    "helm_unet_param_count": (ct.c_size_t, []),
    "helm_unet_layer": (ct.c_int, [ct.c_int, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]),
    "helm_unet_create": (ct.c_int, [ct.POINTER(_P), ct.POINTER(ct.c_double), ct.c_size_t]),
    "helm_unet_create_kind": (ct.c_int, [ct.POINTER(_P), ct.c_int, ct.POINTER(ct.c_double), ct.c_size_t]),
    "helm_unet_param_count_kind": (ct.c_size_t, [ct.c_int]),
    "helm_unet_destroy": (ct.c_int, [_P]),
    "helm_unet_get_weights": (ct.c_int, [_P, ct.POINTER(ct.c_double), ct.c_size_t]),
    "helm_unet_set_weights": (ct.c_int, [_P, _P, ct.c_size_t, _P]),
    "helm_precond_apply": (ct.c_int, [_P, _P, _P, _P, ct.c_int, ct.c_int, _P]),
    "helm_fgmres_solve": (ct.c_int, [_P, _P, _P, _P, ct.c_int, ct.POINTER(helm_solve_opts),
                                     ct.POINTER(helm_solve_info), _P]),
    "helm_train_step": (ct.c_int, [_P, _P, _P, ct.c_double, ct.c_double, ct.c_double, ct.POINTER(ct.c_double),
                                   ct.POINTER(ct.c_double), _P]),
    "helm_loss_grad": (ct.c_int, [_P, _P, _P, ct.c_int, ct.POINTER(ct.c_double), _P, _P]),
    "helm_relres_noalloc": (ct.c_int, [_P, _P, _P, ct.c_int, _P, _P]),
    "helm_unet_layer_forward": (ct.c_int, [_P, ct.c_int, ct.c_int, _P, _P, _P, ct.c_int, ct.c_int, ct.c_int,
                                           ct.POINTER(ct.c_int), _P]),
    "helm_paper_layer_forward": (ct.c_int, [_P, ct.c_int, _P, _P, _P, ct.c_int, ct.c_int, ct.c_int, _P]),
    "helm_unet_get_adam": (ct.c_int, [_P, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double), ct.POINTER(ct.c_int64)]),
    "helm_unet_set_adam": (ct.c_int, [_P, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double), ct.c_int64]),
    "helm_set_wait_budget": (ct.c_int, [ct.c_int64]),
    "helm_inject_fault": (ct.c_int, [ct.c_int, ct.c_int]),
    "helm_solve_history": (ct.c_int, [_P, ct.POINTER(ct.c_double), ct.c_int]),
    "helm_profile_enable": (ct.c_int, [_P, ct.c_int]),
    "helm_profile_read": (ct.c_int, [_P, ct.POINTER(ct.c_double), ct.POINTER(ct.c_int64)]),
    "helm_profile_work": (ct.c_int, [_P, ct.POINTER(ct.c_double)]),
    "helm_launch_count": (ct.c_uint64, []),
    "helm_tuned_tiles": (ct.c_int, [ct.POINTER(ct.c_int), ct.c_int]),
    "helm_tuned_stencil": (ct.c_int, [ct.POINTER(ct.c_int), ct.c_int]),
    "helm_set_stencil_variant": (ct.c_int, [ct.c_int]),
    "helm_last_error": (ct.c_char_p, []),
}
PHASES = ("precond", "stencil", "orth", "lsq", "residual", "update")
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


class HelmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(rc, allow=()):
    if rc != HELM_OK and rc not in allow:
        raise HelmError(rc, _lib.helm_last_error().decode())
    return rc


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ct.c_void_p(s.cuda_stream)


def _dev_ptr(t: torch.Tensor):
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ct.c_void_p(t.data_ptr())


def _batch(t: torch.Tensor, ctx, nrhs, name, dtype=None):
    """Check that t is a contiguous CUDA batch vector with (at least) ctx.npts * nrhs elements."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.numel() < ctx.npts * nrhs:
        raise ValueError(f"{name} holds {t.numel()} values, fewer than npts * nrhs = {ctx.npts * nrhs}")
    return _dev_ptr(t)


def _dtype_code(t: torch.Tensor):
    if t.dtype == torch.complex64:
        return HELM_C64
    if t.dtype == torch.complex128:
        return HELM_C128
    raise TypeError(f"batch vectors must be complex64 or complex128, got {t.dtype}")


@dataclass
class SystemSpec:
    nx: int
    ny: int
    h: float
    width: int
    omega: float
    sigma_max: float = 0.0

    @property
    def Nx(self):
        return self.nx + 2 * self.width

    @property
    def Ny(self):
        return self.ny + 2 * self.width

    @property
    def n(self):
        return self.Nx * self.Ny


class Context:
    """helm_create / helm_destroy: the systems' grids, PMLs, frequencies and velocities."""

    def __init__(self, systems, c: torch.Tensor, stream=None):
        self.systems = list(systems)
        ns = len(self.systems)
        grids = (helm_grid * ns)(*[helm_grid(s.nx, s.ny, s.h) for s in self.systems])
        pmls = (helm_pml * ns)(*[helm_pml(s.width, s.sigma_max) for s in self.systems])
        om = (ct.c_double * ns)(*[s.omega for s in self.systems])
        if c.dtype not in (torch.float64, torch.float32) or c.numel() != sum(s.n for s in self.systems):
            raise ValueError("c must hold sum(Nx*Ny) float32/float64 velocities")
        c = c.contiguous()
        self._h = _P()
        _check(_lib.helm_create(ct.byref(self._h), ns, grids, pmls, om, _dev_ptr(c), int(c.dtype == torch.float64),
                                _stream(stream)))
        self.npts = int(_lib.helm_points(self._h))

    @property
    def handle(self):
        return self._h

    def set_velocity(self, c: torch.Tensor, stream=None):
        """helm_set_velocity: new velocities (same grids) for every system, e.g. the next training batch."""
        if c.dtype not in (torch.float64, torch.float32) or c.numel() != self.npts:
            raise ValueError("c must hold sum(Nx*Ny) float32/float64 velocities")
        c = c.contiguous()
        _check(_lib.helm_set_velocity(self._h, _dev_ptr(c), int(c.dtype == torch.float64), _stream(stream)))

    def close(self):
        if self._h:
            _lib.helm_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def new_vector(self, nrhs=1, dtype=torch.complex128):
        return torch.zeros(self.npts * nrhs, dtype=dtype, device="cuda")


def helm_apply(ctx: Context, x: torch.Tensor, y: torch.Tensor, nrhs=1, adjoint=False, stream=None):
    """y = A x (or A^H x) for complex64/complex128 batch vectors."""
    if x.dtype != y.dtype or x.numel() != ctx.npts * nrhs or y.numel() != x.numel():
        raise ValueError("x, y must be batch vectors of the same dtype and size npts * nrhs")
    f = _lib.helm_apply_adjoint if adjoint else _lib.helm_apply
    _check(f(ctx.handle, _dev_ptr(x), _dev_ptr(y), _dtype_code(x), nrhs, _stream(stream)))
    return y


def helm_apply_fourier(ctx: Context, x: torch.Tensor, y: torch.Tensor, nrhs=1, stream=None):
    """y = A_F x, the Fourier-differentiation operator (helm_apply_fourier in include/helm.h)."""
    if x.dtype != y.dtype or x.numel() != ctx.npts * nrhs or y.numel() != x.numel():
        raise ValueError("x, y must be batch vectors of the same dtype and size npts * nrhs")
    _check(_lib.helm_apply_fourier(ctx.handle, _dev_ptr(x), _dev_ptr(y), _dtype_code(x), nrhs, _stream(stream)))
    return y


def helm_apply_adjoint(ctx, x, y, nrhs=1, stream=None):
    return helm_apply(ctx, x, y, nrhs, adjoint=True, stream=stream)


def helm_relres(ctx: Context, x: torch.Tensor, b: torch.Tensor, nrhs=1, stream=None) -> np.ndarray:
    ncol = len(ctx.systems) * nrhs
    px = _batch(x, ctx, nrhs, "x", torch.complex128)
    pb = _batch(b, ctx, nrhs, "b", torch.complex128)
    out = (ct.c_double * max(ncol, 1))()
    _check(_lib.helm_relres(ctx.handle, px, pb, nrhs, out, _stream(stream)))
    return np.array(out[:])


def helm_relres_noalloc(ctx: Context, x: torch.Tensor, b: torch.Tensor, out: torch.Tensor, nrhs=1, stream=None):
    """Per-column ||b - A x|| / ||b|| into the float64 CUDA tensor `out` (nsys * nrhs entries) without any
    device allocation inside the call; the scratch is a fixed array in the library (see include/helm.h)."""
    ncol = len(ctx.systems) * nrhs
    if out.dtype != torch.float64 or out.numel() < ncol:
        raise ValueError("out must be a float64 CUDA tensor with nsys * nrhs entries")
    px = _batch(x, ctx, nrhs, "x", torch.complex128)
    pb = _batch(b, ctx, nrhs, "b", torch.complex128)
    _check(_lib.helm_relres_noalloc(ctx.handle, px, pb, nrhs, _dev_ptr(out), _stream(stream)))
    return out


def helm_unet_layer_forward(net, layer, in0: torch.Tensor, out: torch.Tensor, B, H, W, in1=None, variant=0,
                            stream=None):
    """One layer of the BF16 network on NHWC bfloat16 CUDA tensors (helm_unet_layer_forward in
    include/helm.h); returns the rows per tile of the row-tile kernel that ran (0: 9-box kernel).
    The tensors' sizes and types are checked here (the library reads and writes them through raw
    pointers)."""
    for t in (in0, out) + ((in1,) if in1 is not None else ()):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("layer tensors must be contiguous CUDA tensors")
    if 0 <= layer <= HELM_LAYER_DEC1B_FINAL and min(B, H, W) >= 1:
        fused = layer == HELM_LAYER_DEC1B_FINAL
        l = 16 if fused else layer
        ci, co, kind = _unet_layers()[l]
        concat = l in (9, 12, 15)  # dec3a, dec2a, dec1a: [up-sampled decoder, skip]
        c0 = 16 if l == 0 else (ci // 2 if concat else ci)  # the input tensor has 16 channels (3 used)
        px = B * H * W
        need = [(in0, "in0", px * c0, torch.bfloat16),
                (out, "out", px * 2 if fused else px * co * (4 if kind == 1 else 1),
                 torch.float32 if fused else torch.bfloat16)]
        if concat and in1 is not None:
            need.append((in1, "in1", px * (ci // 2), torch.bfloat16))
        for t, name, n, dt in need:
            if t.dtype != dt or t.numel() < n:
                raise ValueError(f"helm_unet_layer_forward: {name} must be a {dt} tensor of at least {n} elements")
    ry = ct.c_int()
    _check(_lib.helm_unet_layer_forward(net.handle, layer, variant, _dev_ptr(in0),
                                        _dev_ptr(in1) if in1 is not None else None, _dev_ptr(out), B, H, W,
                                        ct.byref(ry), _stream(stream)))
    return ry.value


HELM_PAPER_LAYER_DEC0_FINAL = 8


def helm_paper_layer_forward(net, layer, in0: torch.Tensor, out: torch.Tensor, B, H, W, in1=None, stream=None):
    """One layer of network kind 1 on NHWC bfloat16 CUDA tensors (helm_paper_layer_forward in
    include/helm.h); H x W is the layer's 5x5 GEMM grid.  The tensors' sizes and types are checked
    here (the library reads and writes them through raw pointers)."""
    for t in (in0, out) + ((in1,) if in1 is not None else ()):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("layer tensors must be contiguous CUDA tensors")
    if 0 <= layer <= HELM_PAPER_LAYER_DEC0_FINAL and min(B, H, W) >= 1:
        fused = layer == HELM_PAPER_LAYER_DEC0_FINAL
        l = 7 if fused else layer
        small, large = B * H * W * 32, B * 4 * H * W * 32  # 32 channels on the H x W / 2H x 2W grid
        need = [(in0, "in0", large if 1 <= l <= 3 else small, torch.bfloat16),
                (out, "out", small if l <= 3 else (B * 4 * H * W * 2 if fused else large),
                 torch.float32 if fused else torch.bfloat16)]
        if in1 is not None:
            need.append((in1, "in1", small, torch.bfloat16))
        for t, name, n, dt in need:
            if t.dtype != dt or t.numel() < n:
                raise ValueError(f"helm_paper_layer_forward: {name} must be a {dt} tensor of at least {n} elements")
    _check(_lib.helm_paper_layer_forward(net.handle, layer, _dev_ptr(in0),
                                         _dev_ptr(in1) if in1 is not None else None, _dev_ptr(out), B, H, W,
                                         _stream(stream)))


def helm_set_wait_budget(cycles: int):
    """Pipeline-wait budget (clock64 cycles) of the TMA/tcgen05 kernels; <= 0 restores the default."""
    _check(_lib.helm_set_wait_budget(int(cycles)))


def helm_inject_fault(site: int, count: int = 1):
    """Arm a host-side fault for the next `count` occurrences of `site` (HELM_FAULT_*)."""
    _check(_lib.helm_inject_fault(int(site), int(count)))


def helm_unet_param_count() -> int:
    return int(_lib.helm_unet_param_count())


def network_kind(nparams: int) -> int:
    """The network kind whose parameter count is `nparams` (helm_unet_param_count_kind: the two
    kinds differ in size); 0 if neither matches (helm_unet_create then rejects the count)."""
    for kind in (0, 1):
        if int(_lib.helm_unet_param_count_kind(kind)) == int(nparams):
            return kind
    return 0


@functools.lru_cache(maxsize=1)
def _unet_layers():
    return tuple(helm_unet_layers())


def helm_unet_layers():
    """[(c_in, c_out, kind)] with kind 0 = 3x3 conv, 1 = 2x2 up-conv, 2 = 1x1 conv, in parameter order."""
    out = []
    for l in range(18):
        a, b, k = ct.c_int(), ct.c_int(), ct.c_int()
        _check(_lib.helm_unet_layer(l, ct.byref(a), ct.byref(b), ct.byref(k)))
        out.append((a.value, b.value, k.value))
    return out


def weight_segments():
    """(count, fan_in, 'w'|'b') per parameter tensor of the library's network, for the seeded generator."""
    seg = []
    for ci, co, k in helm_unet_layers():
        taps = {0: 9, 1: 4, 2: 1}[k]
        fan = ci * {0: 9, 1: 1, 2: 1}[k]
        seg.append((taps * ci * co, fan, "w"))
        seg.append((co, fan, "b"))
    return seg


def paper_weight_segments():
    """(count, fan_in, kind) per parameter tensor of network kind 1 (the paper's variant, see
    include/helm.h), for the seeded generator: 'w' weights, 'b' biases, 's' PReLU slopes."""
    layers = (("down", 5, 32), ("down", 32, 32), ("down", 32, 32), ("down", 32, 32), ("up", 32, 32),
              ("up", 64, 32), ("up", 64, 32), ("up", 64, 32), ("out", 32, 2))
    seg = []
    for kind, ci, co in layers:
        fan = ci * (64 if kind != "out" else 1)
        seg.append((ci * co * (64 if kind != "out" else 1), fan, "w"))
        seg.append((co, fan, "b"))
        if kind != "out":
            seg.append((1, fan, "s"))
    return seg


class UNet:
    """helm_unet_create(_kind) / helm_unet_destroy: network weights (FP64 master) and optimiser state.
    kind 0: the 16/32/64/128 U-Net; kind 1: the paper's variant (include/helm.h)."""

    def __init__(self, weights: np.ndarray, kind=None):
        """kind None: taken from the number of weights (network_kind)."""
        w = np.ascontiguousarray(weights, dtype=np.float64)
        if kind is None:
            kind = network_kind(w.size)
        self._h = _P()
        _check(_lib.helm_unet_create_kind(ct.byref(self._h), int(kind),
                                          w.ctypes.data_as(ct.POINTER(ct.c_double)), w.size))
        self.nparams = w.size
        self.kind = kind

    @property
    def handle(self):
        return self._h

    def weights(self) -> np.ndarray:
        out = np.zeros(self.nparams)
        _check(_lib.helm_unet_get_weights(self._h, out.ctypes.data_as(ct.POINTER(ct.c_double)), out.size))
        return out

    def adam_state(self):
        """(m, v, step) of the AdamW optimiser (helm_unet_get_adam)."""
        m, v, st = np.zeros(self.nparams), np.zeros(self.nparams), ct.c_int64()
        _check(_lib.helm_unet_get_adam(self._h, m.ctypes.data_as(ct.POINTER(ct.c_double)),
                                       v.ctypes.data_as(ct.POINTER(ct.c_double)), ct.byref(st)))
        return m, v, st.value

    def set_adam_state(self, m, v, step):
        """Restore the AdamW moments and step count (helm_unet_set_adam)."""
        m = np.ascontiguousarray(m, np.float64)
        v = np.ascontiguousarray(v, np.float64)
        if m.size != self.nparams or v.size != self.nparams:
            raise ValueError("moments must have one value per parameter")
        _check(_lib.helm_unet_set_adam(self._h, m.ctypes.data_as(ct.POINTER(ct.c_double)),
                                       v.ctypes.data_as(ct.POINTER(ct.c_double)), int(step)))

    def set_weights(self, theta: torch.Tensor, stream=None):
        """helm_unet_set_weights: replace the weights from a CUDA float64 tensor of nparams values."""
        if theta.dtype != torch.float64 or not theta.is_cuda or theta.numel() != self.nparams:
            raise ValueError("theta must be a CUDA float64 tensor with one value per parameter")
        _check(_lib.helm_unet_set_weights(self._h, _dev_ptr(theta.contiguous()), self.nparams, _stream(stream)))

    def close(self):
        if self._h:
            _lib.helm_unet_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def helm_precond_apply(ctx: Context, net: UNet, v: torch.Tensor, z: torch.Tensor, nrhs=1, stream=None):
    if v.dtype != z.dtype or v.numel() != ctx.npts * nrhs or z.numel() != v.numel():
        raise ValueError("v, z must be batch vectors of the same dtype and size npts * nrhs")
    _check(_lib.helm_precond_apply(ctx.handle, net.handle, _dev_ptr(v), _dev_ptr(z), _dtype_code(v), nrhs,
                                   _stream(stream)))
    return z


ORTH = {"cgs2": 0, "dcgs2": 1}


def helm_fgmres_solve(ctx: Context, net, b: torch.Tensor, x: torch.Tensor, nrhs=1, m=30, tol=1e-6,
                      mixed=True, max_restarts=100, max_outer=100, inner_tol=1e-4, orth="cgs2", stream=None,
                      raise_on=False):
    """Solve A x = b (complex128 batch vectors; x holds x0 on entry).  Returns (status, [info dict per column])."""
    if b.dtype != torch.complex128 or x.dtype != torch.complex128:
        raise TypeError("b and x are complex128 batch vectors")
    if b.numel() != ctx.npts * nrhs or x.numel() != b.numel():
        raise ValueError("b, x must have npts * nrhs entries")
    ncol = len(ctx.systems) * nrhs
    opts = helm_solve_opts(m, max_restarts, max_outer, tol, inner_tol, int(bool(mixed)), ORTH[orth])
    info = (helm_solve_info * ncol)()
    rc = _lib.helm_fgmres_solve(ctx.handle, net.handle if net is not None else None, _dev_ptr(b), _dev_ptr(x),
                                nrhs, ct.byref(opts), info, _stream(stream))
    _check(rc, allow=() if raise_on else (HELM_NOT_CONVERGED, HELM_BREAKDOWN, HELM_NAN, HELM_TIMEOUT))
    cols = [dict(iters=i.iters, restarts=i.restarts, outer=i.outer, relres_true=i.relres_true,
                 relres_est=i.relres_est, status=STATUS_NAMES.get(i.status, i.status)) for i in info]
    return rc, cols


def helm_solve_history(ctx: Context) -> np.ndarray:
    """Per-iteration residual estimates (relative to ||b||) of column 0 of the last solve."""
    n = _lib.helm_solve_history(ctx.handle, None, 0)
    buf = (ct.c_double * max(n, 1))()
    _lib.helm_solve_history(ctx.handle, buf, n)
    return np.array(buf[:n])


def helm_train_step(ctx: Context, net: UNet, b: torch.Tensor, lr=1e-3, wd=0.01, clip=1.0, stream=None):
    """One AdamW step on the batch loss (eqs. 8-9); b is a complex64 batch vector, one source per system.
    Returns (loss before the update, gradient norm before clipping)."""
    if b.dtype != torch.complex64 or b.numel() != ctx.npts:
        raise ValueError("b must be a complex64 batch vector with one right-hand side per system")
    loss, gn = ct.c_double(), ct.c_double()
    _check(_lib.helm_train_step(ctx.handle, net.handle, _dev_ptr(b), lr, wd, clip, ct.byref(loss), ct.byref(gn),
                                _stream(stream)))
    return loss.value, gn.value


def helm_loss_grad(ctx: Context, net: UNet, b: torch.Tensor, stream=None):
    """Loss (eq. 9, batch mean) and its FP64 gradient w.r.t. the flat parameter vector (CUDA tensor).
    complex64 b differentiates the BF16 network path, complex128 b the FP64 path."""
    if b.numel() != ctx.npts:
        raise ValueError("b must be a batch vector with one right-hand side per system")
    g = torch.zeros(net.nparams, dtype=torch.float64, device="cuda")
    loss = ct.c_double()
    _check(_lib.helm_loss_grad(ctx.handle, net.handle, _dev_ptr(b), _dtype_code(b), ct.byref(loss), _dev_ptr(g),
                               _stream(stream)))
    return loss.value, g


class HelmholtzLoss(torch.autograd.Function):
    """Eq. 9 as a differentiable function of the flat parameter vector theta (CUDA float64):
    forward loads theta into `net` and returns the batch-mean loss; backward returns the library's
    gradient (adjoint stencil A^H and conv backward kernels), scaled by the incoming gradient.
    Usage: loss = HelmholtzLoss.apply(theta, ctx, net, b); loss.backward()."""

    @staticmethod
    def forward(fctx, theta, ctx, net, b):
        net.set_weights(theta.detach())
        loss, grad = helm_loss_grad(ctx, net, b)
        fctx.save_for_backward(grad)
        return torch.tensor(loss, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(fctx, gout):
        (grad,) = fctx.saved_tensors
        return gout * grad, None, None, None


def helm_profile_enable(ctx: Context, on=True):
    """Enable (and reset) or disable the solver's per-phase CUDA-event timers."""
    _check(_lib.helm_profile_enable(ctx.handle, int(bool(on))))


def helm_profile_read(ctx: Context):
    """{phase: (milliseconds, intervals)} accumulated since helm_profile_enable."""
    ms = (ct.c_double * len(PHASES))()
    cnt = (ct.c_int64 * len(PHASES))()
    _check(_lib.helm_profile_read(ctx.handle, ms, cnt))
    return {p: (ms[i], cnt[i]) for i, p in enumerate(PHASES)}


def helm_profile_work(ctx: Context):
    """{phase: algorithmic flops (precond) or bytes (other phases)} issued since helm_profile_enable."""
    w = (ct.c_double * len(PHASES))()
    _check(_lib.helm_profile_work(ctx.handle, w))
    return {p: w[i] for i, p in enumerate(PHASES)}


def helm_tuned_tiles():
    """Rows per tile the autotuner chose per row-conv layer shape: list of dicts."""
    buf = (ct.c_int * (6 * 256))()
    n = _lib.helm_tuned_tiles(buf, 256)
    keys = ("c_out", "slices", "images", "H", "W", "rows_per_tile")
    return [dict(zip(keys, buf[6 * k: 6 * k + 6])) for k in range(n)]


def helm_set_stencil_variant(variant: int):
    """Force FP32 stencil tile candidate `variant` (1..4) for later launches; 0 restores tuning."""
    _check(_lib.helm_set_stencil_variant(int(variant)))


def helm_tuned_stencil():
    """Tile shape the autotuner chose per FP32 stencil grid shape: list of dicts."""
    buf = (ct.c_int * (6 * 256))()
    n = _lib.helm_tuned_stencil(buf, 256)
    keys = ("Nx", "Ny", "nrhs", "adjoint", "rows_per_tile", "stages")
    return [dict(zip(keys, buf[6 * k: 6 * k + 6])) for k in range(n)]


def helm_launch_count() -> int:
    """Kernels launched by libhelm in this process so far."""
    return int(_lib.helm_launch_count())
