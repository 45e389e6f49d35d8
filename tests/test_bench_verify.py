"""The benchmark's verification pool (bench_verify) on the CPU: its workers
regenerate each product's operands exactly as synth.batch_operands drew
them, and their digests are those of the oracle's exact product."""
import numpy as np

import synth
from bench_verify import OraclePool, batch_jobs, digest
from oracle import exact as E


def test_pool_digests_equal_the_oracle_products():
    seed = synth.SEED_BASE + 77
    na = np.array([1, 3, 700, 5000, 64])
    nb = np.array([1, 2000, 700, 17, 64])
    dists = ["uniform", "ff", "uniform", "uniform", "zero"]
    a_pool, b_pool, a_off, b_off, _ = synth.batch_operands(seed, na, nb, dists)
    jobs = batch_jobs(seed, na, nb, dists) + [("pair", seed, 300, 200, "uniform", "schoolbook"),
                                              ("pair", seed, 4096, 4096, "ff", "ntt")]
    with OraclePool(2) as pool:
        got = pool.digests(jobs)
    for p in range(len(na)):
        a = a_pool[a_off[p]:a_off[p] + na[p]]
        b = b_pool[b_off[p]:b_off[p] + nb[p]]
        assert got[p] == digest(E.product(a, b))
    a, b = synth.operand_pair(seed, 300, 200)
    assert got[-2] == digest(E.long_mul(a, b))
    assert got[-1] == digest(E.product(*synth.operand_pair(seed, 4096, 4096, "ff")))
    # a single changed digit changes the digest
    z = E.product(a, b)
    z[17] ^= 1
    assert digest(z) != got[-2]
