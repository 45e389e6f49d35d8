"""Helpers for the GPU tests: device buffers through torch, calls through the C ABI."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1006_0405_gb300 import abi  # noqa: E402


def dev(x: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


class Plan:
    def __init__(self, max_na, max_nb, max_products=0, prec=abi.SSMUL_PREC_FP64):
        self.h = abi.ssmul_plan(max_na, max_nb, max_products, prec, 0)

    def close(self):
        if self.h:
            abi.ssmul_plan_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def mul(self, a: np.ndarray, b: np.ndarray):
        da, db = dev(a), dev(b)
        dz = torch.full((len(a) + len(b),), 0xA5, dtype=torch.uint8, device="cuda")
        s, r = abi.ssmul_mul(self.h, da.data_ptr(), len(a), db.data_ptr(), len(b), dz.data_ptr())
        return s, r, dz.cpu().numpy()

    def mul_intervals(self, a, b, prec):
        da, db = dev(a), dev(b)
        L = len(a) + len(b) - 1
        dz = torch.zeros(len(a) + len(b), dtype=torch.uint8, device="cuda")
        div = torch.zeros(2 * L, dtype=torch.float64, device="cuda")
        s, r = abi.ssmul_debug_mul_intervals(self.h, da.data_ptr(), len(a), db.data_ptr(), len(b),
                                             dz.data_ptr(), prec, div.data_ptr())
        iv = div.cpu().numpy().reshape(L, 2)
        return s, r, dz.cpu().numpy(), iv[:, 0], iv[:, 1]

    def twiddles(self, f32=False, log_max=24, odd=1):
        """(K, cos_lo, cos_hi, sin_lo, sin_hi) of the table Ntab = odd * 2^K (odd 1, 3 or 5)."""
        cap = 4 * ((1 << log_max) // 8 + 1)
        buf = np.zeros(cap, np.float64)
        flags = int(f32) | {1: 0, 3: 2, 5: 4}[odd]
        s, ln = abi.ssmul_debug_twiddles(self.h, flags, buf.ctypes.data, cap)
        assert s == abi.SSMUL_OK
        m = (odd << ln) // 8 + 1
        t = buf[:4 * m].reshape(m, 4)
        return ln, t[:, 0], t[:, 1], t[:, 2], t[:, 3]


def batched(plan: Plan, pairs):
    """Run a list of (a, b) through ssmul_mul_batched; returns (status, results, digits list)."""
    na = [len(a) for a, _ in pairs]
    nb = [len(b) for _, b in pairs]
    a_pool = np.concatenate([a for a, _ in pairs])
    b_pool = np.concatenate([b for _, b in pairs])
    a_off = np.concatenate([[0], np.cumsum(na)[:-1]])
    b_off = np.concatenate([[0], np.cumsum(nb)[:-1]])
    nz = np.array(na) + np.array(nb)
    z_off = np.concatenate([[0], np.cumsum(nz)[:-1]])
    da, db = dev(a_pool), dev(b_pool)
    dz = torch.full((int(nz.sum()),), 0xA5, dtype=torch.uint8, device="cuda")
    res = (abi.ssmul_result * len(pairs))()
    dres = torch.zeros(ctypes.sizeof(res), dtype=torch.uint8, device="cuda")
    descs = [(int(a_off[i]), int(b_off[i]), int(z_off[i]), na[i], nb[i]) for i in range(len(pairs))]
    s = abi.ssmul_mul_batched(plan.h, descs, da.data_ptr(), db.data_ptr(), dz.data_ptr(),
                              dres.data_ptr())
    torch.cuda.synchronize()
    host = dres.cpu().numpy()
    ctypes.memmove(res, host.ctypes.data, ctypes.sizeof(res))
    z = dz.cpu().numpy()
    digits = [z[z_off[i]:z_off[i] + nz[i]] for i in range(len(pairs))]
    return s, list(res), digits
