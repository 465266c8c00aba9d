"""Closed-form attention operation counts of appendix A (One-to-Many Attention).

TEST INFRASTRUCTURE ONLY (see quark_oracle.py).

The appendix counts multiply-accumulates ("flops" in its tables) for one query
attending over N inputs with h heads of model width d_k:
  standard cross attention   (2N + 1) d_k^2 + N d_k + d_k^2
  one-to-many attention      h d_k^2 + N h d_k + h d_k^2
Neither count includes the N-term weighted sum of the values; `with_weighted_sum`
adds it (N d_k and N h d_k respectively) for the per-element MAC accounting.
"""


def standard_macs(N: int, d_k: int, h: int = 1, with_weighted_sum: bool = False) -> int:
    n = (2 * N + 1) * d_k * d_k + N * d_k + d_k * d_k
    return n + (N * d_k if with_weighted_sum else 0)


def one_to_many_macs(N: int, d_k: int, h: int, with_weighted_sum: bool = False) -> int:
    n = h * d_k * d_k + N * h * d_k + h * d_k * d_k
    return n + (N * h * d_k if with_weighted_sum else 0)
