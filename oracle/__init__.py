"""CPU oracle for the interval Schoenhage-Strassen multiplier.

TEST INFRASTRUCTURE ONLY.  Only the tests, `__graft_entry__.smoke()` and the
CPU-baseline / reference legs of `bench.py` import anything from here.  The
product path (the `paper_1006_0405_gb300` package and its CUDA library)
never imports, links or calls this package, and the two share no code.

Modules
  exact       exact integer results: long multiplication (Section 2.1),
              convolution coefficients (Section 2.1), carry (Section 2.4),
              an NTT exact convolution for large sizes, residues mod primes.
  interval    IEEE directed rounding, real and rectangular complex interval
              arithmetic (Section 2.5) and the unique-integer isolation
              decision (Section 1, Section 2.5).
  twiddle     rigorous enclosures of the roots of unity omega^j (Section 2.2)
              from exact integer arithmetic.
  interval_ss the paper's rigorous algorithm end to end: interval radix-2 FFT
              (Section 2.2), fast convolution (Section 2.3), isolation and
              carry (Section 2.4), in the paper's order.

Parity status of each function is listed in its module header.
"""
