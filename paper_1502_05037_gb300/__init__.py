"""GB300 SARA/SDMM radio-interferometric imaging (arXiv:1502.05037).

Thin Python layer over the C ABI of libpurify.so: the functions below carry
the C names and only marshal arguments. Arrays are torch tensors (device or
host) or NumPy arrays (host) of the plan's dtype; complex arrays are
torch.complex64/complex128 (or interleaved real pairs).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (PURIFY_F32, PURIFY_F64, PurifyError, check, load, purify_kernel_time, purify_plan_desc,
                   purify_pd_params, purify_plan_info, purify_sdmm_params, purify_sdmm_stats)

__all__ = [
    "Plan", "purify_plan_create", "purify_plan_destroy", "purify_phi", "purify_phi_adj", "purify_phi_normal",
    "purify_fft2",
    "purify_psi", "purify_psi_adj", "purify_op_norm_sq", "purify_sdmm_solve", "purify_sdmm_iterate",
    "purify_reweight",
    "purify_coef_std", "purify_launch_count", "PurifyError", "PURIFY_F32", "PURIFY_F64",
]


def _ptr(a) -> int | None:
    """Raw data pointer of a torch tensor or NumPy array (must be contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _nbytes(a) -> int | None:
    if isinstance(a, np.ndarray):
        return a.nbytes
    if hasattr(a, "numel") and hasattr(a, "element_size"):
        return a.numel() * a.element_size()
    return None


def _need(plan, a, values, name: str, cplx: bool = False):
    """The C calls take raw pointers and cannot see the caller's buffer
    sizes: refuse a buffer smaller than the `values` real (or complex)
    elements of the plan's precision that the call reads or writes, instead
    of letting the device touch memory past its end."""
    if a is None:
        return
    have = _nbytes(a)
    need = int(values) * (4 if plan.dtype == PURIFY_F32 else 8) * (2 if cplx else 1)
    if have is not None and have < need:
        raise ValueError(f"{name} holds {have} bytes; this plan's call needs {need}")


def _need_eps(plan, eps):
    if eps is not None and np.asarray(eps).size < plan.info.R:
        raise ValueError(f"eps needs one bound per block ({plan.info.R})")


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Plan:
    """Owns a purify_plan handle; see purify_plan_create for the fields."""

    def __init__(self, nx, ny, u, v, kb_width=6, levels=4, block_offsets=None, oversample=2.0, kb_beta=0.0,
                 basis_mask=0, dtype=PURIFY_F32, stream=None, tile=0, grid_mode=0):
        lib = load()
        M = int(u.numel() if hasattr(u, "numel") else np.asarray(u).size)
        self._keep = [u, v]
        offs = None
        R = 1
        if block_offsets is not None:
            offs_np = np.ascontiguousarray(np.asarray(block_offsets, dtype=np.int64))
            self._keep.append(offs_np)
            R = offs_np.size - 1
            offs = offs_np.ctypes.data_as(C.POINTER(C.c_int64))
        d = purify_plan_desc(nx=nx, ny=ny, M=M, u=_ptr(u), v=_ptr(v), R=R, block_offsets=offs,
                             kb_width=kb_width, oversample=oversample, kb_beta=kb_beta, levels=levels,
                             basis_mask=basis_mask, dtype=dtype, stream=_stream_ptr(stream), tile=tile,
                             grid_mode=grid_mode)
        h = C.c_void_p()
        check(lib.purify_plan_create(C.byref(d), C.byref(h)))
        self.handle = h
        self._keep = None
        self.dtype = dtype
        info = purify_plan_info()
        check(lib.purify_plan_get_info(h, C.byref(info)))
        self.info = info

    def close(self):
        if getattr(self, "handle", None):
            check(load().purify_plan_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        check(load().purify_plan_set_stream(self.handle, _stream_ptr(stream)))


# ------------------------------------------------- C-named thin wrappers
def purify_plan_create(**kw) -> Plan:
    return Plan(**kw)


def purify_plan_destroy(plan: Plan):
    plan.close()


def purify_phi(plan: Plan, x, y):
    _need(plan, x, plan.info.N, "x")
    _need(plan, y, plan.info.M, "y", cplx=True)
    check(load().purify_phi(plan.handle, _ptr(x), _ptr(y)))


def purify_phi_adj(plan: Plan, y, x):
    _need(plan, y, plan.info.M, "y", cplx=True)
    _need(plan, x, plan.info.N, "x", cplx=True)
    check(load().purify_phi_adj(plan.handle, _ptr(y), _ptr(x)))


def purify_phi_normal(plan: Plan, x, out):
    """out = Re Phi^H Phi x (real images), the solver's normal operator."""
    _need(plan, x, plan.info.N, "x")
    _need(plan, out, plan.info.N, "out")
    check(load().purify_phi_normal(plan.handle, _ptr(x), _ptr(out)))


def purify_fft2(plan: Plan, grid, inverse: bool = False):
    _need(plan, grid, plan.info.Kx * plan.info.Ky, "grid", cplx=True)
    check(load().purify_fft2(plan.handle, _ptr(grid), int(bool(inverse))))


def purify_psi(plan: Plan, c, x):
    _need(plan, c, plan.info.D, "c")
    _need(plan, x, plan.info.N, "x")
    check(load().purify_psi(plan.handle, _ptr(c), _ptr(x)))


def purify_psi_adj(plan: Plan, x, c):
    _need(plan, x, plan.info.N, "x")
    _need(plan, c, plan.info.D, "c")
    check(load().purify_psi_adj(plan.handle, _ptr(x), _ptr(c)))


def purify_op_norm_sq(plan: Plan, iters: int = 100) -> float:
    out = C.c_double()
    check(load().purify_op_norm_sq(plan.handle, iters, C.byref(out)))
    return out.value


def _int32_seq(seq):
    if seq is None:
        return None, None
    a = np.ascontiguousarray(np.asarray(seq, dtype=np.int32))
    return a, a.ctypes.data_as(C.POINTER(C.c_int32))


def purify_sdmm_solve(plan: Plan, y, eps, x, w=None, max_iter=200, cg_iters=10, cg_tol=0.0, gamma=0.0, nu=0.0,
                      rel_obj_tol=0.0, eps_tol=0.0, check_every=0, resume=False, toeplitz=False,
                      block_groups=0, group_seq=None, raise_on_error=True):
    """Solve problem (3); x is updated in place. Returns purify_sdmm_stats.
    block_groups / group_seq: stochastic block-subset iterations (group_seq
    holds max_iter group indices)."""
    _need(plan, y, plan.info.M, "y", cplx=True)
    _need(plan, w, plan.info.D, "w")
    _need(plan, x, plan.info.N, "x")
    _need_eps(plan, eps)
    eps_np = None
    eps_ptr = None
    if eps is not None:
        eps_np = np.ascontiguousarray(np.asarray(eps, dtype=np.float64))
        eps_ptr = eps_np.ctypes.data_as(C.POINTER(C.c_double))
    seq_np, seq_ptr = _int32_seq(group_seq)
    if seq_np is not None and seq_np.size < max_iter:
        raise ValueError("group_seq needs max_iter entries")
    prm = purify_sdmm_params(max_iter=max_iter, cg_iters=cg_iters, cg_tol=cg_tol, gamma=gamma, nu=nu,
                             rel_obj_tol=rel_obj_tol, eps_tol=eps_tol, check_every=check_every,
                             resume=int(bool(resume)), toeplitz=int(bool(toeplitz)), block_groups=block_groups,
                             group_seq=seq_ptr)
    st = purify_sdmm_stats()
    status = load().purify_sdmm_solve(plan.handle, _ptr(y), eps_ptr, _ptr(w), _ptr(x), C.byref(prm), C.byref(st))
    if raise_on_error:
        check(status)
    return st


def purify_pd_solve(plan: Plan, y, eps, x, w=None, iters=200, tau=0.0, sigma=0.0, nu=0.0):
    """Primal-dual (Chambolle-Pock) iterations for problem (3); x is updated
    in place. Returns purify_sdmm_stats."""
    _need(plan, y, plan.info.M, "y", cplx=True)
    _need(plan, w, plan.info.D, "w")
    _need(plan, x, plan.info.N, "x")
    _need_eps(plan, eps)
    eps_np = np.ascontiguousarray(np.asarray(eps, dtype=np.float64))
    prm = purify_pd_params(iters=iters, tau=tau, sigma=sigma, nu=nu)
    st = purify_sdmm_stats()
    check(load().purify_pd_solve(plan.handle, _ptr(y), eps_np.ctypes.data_as(C.POINTER(C.c_double)), _ptr(w),
                                 _ptr(x), C.byref(prm), C.byref(st)))
    return st


def purify_sdmm_iterate(plan: Plan, iters: int):
    """Advance the plan's current SDMM state by `iters` iterations (async)."""
    check(load().purify_sdmm_iterate(plan.handle, int(iters)))


def purify_sdmm_iterate_groups(plan: Plan, iters: int, groups=None):
    """Advance a block-group solve by `iters` iterations, iteration i on group
    groups[i] (None: round-robin); asynchronous."""
    seq_np, seq_ptr = _int32_seq(groups)
    if seq_np is not None and seq_np.size < iters:
        raise ValueError("groups needs iters entries")
    check(load().purify_sdmm_iterate_groups(plan.handle, int(iters), seq_ptr))


class Batch:
    """Several plans advanced together (purify_batch_*); `stream` must be a
    non-default torch.cuda.Stream (graph capture needs one)."""

    def __init__(self, plans, stream):
        lib = load()
        self.plans = list(plans)
        arr = (C.c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        h = C.c_void_p()
        check(lib.purify_batch_create(arr, len(self.plans), _stream_ptr(stream), C.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            check(load().purify_batch_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def purify_batch_create(plans, stream) -> Batch:
    return Batch(plans, stream)


def purify_batch_iterate(batch: Batch, iters: int):
    check(load().purify_batch_iterate(batch.handle, int(iters)))


def purify_batch_destroy(batch: Batch):
    batch.close()


def purify_reweight(plan: Plan, x, rho: float, w):
    _need(plan, x, plan.info.N, "x")
    _need(plan, w, plan.info.D, "w")
    check(load().purify_reweight(plan.handle, _ptr(x), float(rho), _ptr(w)))


def purify_coef_std(plan: Plan, x) -> float:
    _need(plan, x, plan.info.N, "x")
    out = C.c_double()
    check(load().purify_coef_std(plan.handle, _ptr(x), C.byref(out)))
    return out.value


def purify_psi_adj_static(x, c, nx: int, ny: int, levels: int, basis_mask: int = 0, dtype: int = PURIFY_F32,
                          stream=None):
    """Psi^dagger without a plan and without any device allocation (device
    pointers only; see include/purify.h for the size limit and sharing).
    The C side cannot see buffer sizes, so they are checked here: x holds
    nx * ny and c q * nx * ny values of `dtype`, q the number of bases."""
    mask = basis_mask if basis_mask else 0x1FF
    q = bin(mask & 0x1FF).count("1")
    itemsize = 4 if dtype == PURIFY_F32 else 8
    for name, a, n in (("x", x, nx * ny), ("c", c, q * nx * ny)):
        if hasattr(a, "numel"):
            size, isz = a.numel(), a.element_size()
            floating = a.is_floating_point()
        else:
            arr = np.asarray(a)
            size, isz, floating = arr.size, arr.itemsize, arr.dtype.kind == "f"
        if size != n or isz != itemsize or not floating:
            raise ValueError(f"{name} must hold {n} {'float32' if itemsize == 4 else 'float64'} values")
    check(load().purify_psi_adj_static(_ptr(x), _ptr(c), nx, ny, levels, basis_mask, dtype, _stream_ptr(stream)))


def purify_conv2d(x, w, bias, out, k: int, relu: bool = False, stream=None):
    """Tensor-core BF16 convolution (see include/purify.h): x [B][H][W][Cin],
    w [Cout][k][k][Cin], out [B][H][W][Cout], FP32 device tensors."""
    B, H, W, Cin = x.shape
    Cout = w.shape[0]
    check(load().purify_conv2d(_ptr(x), B, H, W, Cin, _ptr(w), _ptr(bias), Cout, k, int(bool(relu)), _ptr(out),
                               _stream_ptr(stream)))


class Unet:
    """The learned warm-start network (purify_unet_*). Tensors are FP32
    device arrays [B][H][W]."""

    def __init__(self, H, W, levels=4, base=32, max_batch=8, seed=0, stream=None):
        lib = load()
        h = C.c_void_p()
        check(lib.purify_unet_create(H, W, levels, base, max_batch, seed, _stream_ptr(stream), C.byref(h)))
        self.handle = h
        self.H, self.W, self.levels, self.base, self.max_batch = H, W, levels, base, max_batch
        self.num_params = int(lib.purify_unet_num_params(h))

    def close(self):
        if getattr(self, "handle", None):
            check(load().purify_unet_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self, out):
        check(load().purify_unet_get_params(self.handle, _ptr(out)))

    def set_params(self, p):
        check(load().purify_unet_set_params(self.handle, _ptr(p)))

    def forward(self, x, y):
        check(load().purify_unet_forward(self.handle, _ptr(x), _ptr(y), int(x.shape[0])))

    def gradients(self, x, target, grads=None) -> float:
        loss = C.c_double()
        check(load().purify_unet_gradients(self.handle, _ptr(x), _ptr(target), int(x.shape[0]), _ptr(grads),
                                           C.byref(loss)))
        return loss.value

    def train_step(self, x, target, lr, want_loss=False):
        loss = C.c_double()
        check(load().purify_unet_train_step(self.handle, _ptr(x), _ptr(target), int(x.shape[0]), float(lr),
                                            C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None


def purify_timing_enable(plan: Plan, enable: bool = True):
    check(load().purify_timing_enable(plan.handle, int(bool(enable))))


def purify_timing_read(plan: Plan, reset: bool = True) -> dict:
    lib = load()
    buf = (purify_kernel_time * 64)()
    n = lib.purify_timing_read(plan.handle, buf, 64, int(bool(reset)))
    if n < 0:
        check(1)
    return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms) for i in range(min(n, 64))}


def purify_launch_count() -> int:
    return int(load().purify_launch_count())
