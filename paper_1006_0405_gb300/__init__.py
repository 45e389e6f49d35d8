"""Verified integer multiplication by complex interval FFT convolution on GB300.

The hot path (interval FFTs with directed rounding, pointwise products,
unique-integer isolation and the carry scan) runs in the CUDA library
libssmul.so behind the C ABI of include/ssmul.h; this package holds its
build step (`build`), its ctypes binding (`abi`) and a small torch-facing
convenience layer (`Multiplier`).  PyTorch only provides device memory and
streams.
"""
from __future__ import annotations

from . import abi
from .abi import (SSMUL_OK, SSMUL_ISOLATION_FAILED, SSMUL_CONTAINMENT_FAILED,  # noqa: F401
                  SSMUL_PREC_FP64, SSMUL_PREC_FP32, SSMUL_PREC_LADDER, SsmulError)

__all__ = ["abi", "Multiplier", "SSMUL_OK", "SSMUL_PREC_FP64", "SSMUL_PREC_FP32",
           "SSMUL_PREC_LADDER"]


class Multiplier:
    """A plan plus torch-allocated device buffers.

    mul(a, b) takes uint8 CUDA tensors of little-endian base-256 digits and
    returns (z, result) with z the na + nb product digits (zero-filled unless
    result.status == SSMUL_OK).
    """

    def __init__(self, max_na: int, max_nb: int, max_products: int = 0,
                 prec: int = SSMUL_PREC_FP64, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("ssmul needs a CUDA device; there is no CPU path")
        self._torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.plan = abi.ssmul_plan(max_na, max_nb, max_products, prec, self.stream.cuda_stream)
        self.max_na, self.max_nb, self.prec = max_na, max_nb, prec

    def close(self):
        if getattr(self, "plan", None):
            abi.ssmul_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def mul(self, a, b, out=None):
        torch = self._torch
        assert a.dtype == torch.uint8 and b.dtype == torch.uint8 and a.is_cuda and b.is_cuda
        a, b = a.contiguous(), b.contiguous()
        z = out if out is not None else torch.empty(a.numel() + b.numel(), dtype=torch.uint8,
                                                    device=a.device)
        s, r = abi.ssmul_mul(self.plan, a.data_ptr(), a.numel(), b.data_ptr(), b.numel(),
                             z.data_ptr())
        if s not in (abi.SSMUL_OK, abi.SSMUL_ISOLATION_FAILED, abi.SSMUL_CONTAINMENT_FAILED,
                     abi.SSMUL_TIMEOUT):
            raise SsmulError(s, "ssmul_mul")
        return z, r
