"""Bit-exact verification of benchmark products against the CPU oracle.

A product counts as verified when its status is SSMUL_OK and its digits
equal the oracle's exact product (the convolution of Section 2.1 by the
oracle's NTT, then the carry of Section 2.4; long multiplication, Section
2.1, where a workload names schoolbook).  For batches of thousands of
products the oracle runs in a pool of worker processes started with the
"spawn" method (never forked from a process that holds a CUDA context),
one oracle thread per worker.  A worker regenerates its product's operands
from the workload's seed with `synth` (the generator the GPU inputs came
from) and returns the SHA-256 digest of the exact digits; the parent
compares it with the digest of the digits the GPU returned, so equal
digests mean equal bytes without moving the digit arrays between processes.
"""
from __future__ import annotations

import hashlib
import multiprocessing as mp
import os

import numpy as np

import synth


def digest(z) -> bytes:
    return hashlib.sha256(np.ascontiguousarray(z, dtype=np.uint8).tobytes()).digest()


def _init_worker():
    from oracle import exact as E
    E.lib()


def _exact_digest(job) -> bytes:
    """job: ("batch", seed, p, na, nb, dist) for product p of
    synth.batch_operands(seed, ...), or ("pair", seed, na, nb, dist, how)
    for synth.operand_pair(seed, na, nb, dist); how: "ntt" or "schoolbook"."""
    from oracle import exact as E
    if job[0] == "batch":
        _, seed, p, na, nb, dist = job
        a, b = synth.operand_pair(synth._substream(seed, 1000 + p), na, nb, dist)
        how = "ntt"
    else:
        _, seed, na, nb, dist, how = job
        a, b = synth.operand_pair(seed, na, nb, dist)
    if how == "schoolbook":
        z = E.long_mul(a, b)
    else:
        z = E.carry(E.conv_ntt(a, b), na + nb)
    return digest(z)


class OraclePool:
    """A spawn-started pool of oracle workers (one per host core, each with
    one OpenMP thread)."""

    def __init__(self, processes: int | None = None):
        self.processes = processes or os.cpu_count() or 1
        old = os.environ.get("OMP_NUM_THREADS")
        os.environ["OMP_NUM_THREADS"] = "1"         # inherited by the spawned workers
        try:
            self.pool = mp.get_context("spawn").Pool(self.processes, initializer=_init_worker)
        finally:
            if old is None:
                del os.environ["OMP_NUM_THREADS"]
            else:
                os.environ["OMP_NUM_THREADS"] = old

    def digests(self, jobs) -> list:
        jobs = list(jobs)
        # large products first, so no worker is left with one at the end
        order = sorted(range(len(jobs)), key=lambda i: -_weight(jobs[i]))
        out = [None] * len(jobs)
        for i, d in zip(order, self.pool.imap(_exact_digest, [jobs[i] for i in order],
                                                chunksize=4)):
            out[i] = d
        return out

    def close(self):
        self.pool.close()
        self.pool.join()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _weight(job) -> int:
    return (job[3] + job[4]) if job[0] == "batch" else (job[2] + job[3])


def batch_jobs(seed: int, na, nb, dists) -> list:
    return [("batch", int(seed), p, int(na[p]), int(nb[p]), str(dists[p])) for p in range(len(na))]


def count_verified(results, digits, expected_digests, ok_status: int = 0):
    """(verified products, verified digits): status ok_status and digest equal."""
    n = d = 0
    for r, z, e in zip(results, digits, expected_digests):
        if r.status == ok_status and digest(z) == e:
            n += 1
            d += len(z)
    return n, d
