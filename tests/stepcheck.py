"""Per-step checks of GPU iterates against Algorithm 1 (test infrastructure).

Every GPU loop can log i_k and x_k, the iterate step k selects from.  From
those logs the checks here replay each step in binary64:

* r_k = bt - At x_k is recomputed exactly enough (FP64) from the GPU's own
  x_k, and a bound B_k,j on |r_gpu,k,j - r_k,j| -- how far the residual the
  GPU actually scored can be from it -- is derived from the arithmetic of
  the residual path (below);
* selection (Algorithm 1, i_k = argmax_j r_j^2 / ||At_j||^2 over non-zero
  rows): i_k is admissible, i.e. no row's lower key bound exceeds i_k's
  upper bound.  A step is "forced" when i_k's lower bound exceeds every
  other row's upper bound: the bound then proves i_k is THE maximiser;
* projection (Algorithm 1, x_{k+1} = x_k + r_{i_k} / ||At_{i_k}||^2 At_{i_k}^T):
  x_{k+1} - x_k equals the exact step to within the same bound plus the
  rounding of the update;
* the oracle's own selection, run from the GPU's x_k (one step of
  ``oracle.mwrk`` with x0 = x_k), must pick i_k unless its pick is also
  admissible (a near-tie that the rounding may decide either way).

Bounds on the residual the GPU scores (u = 2^-24, the FP32 unit roundoff):

* GEMV path (r recomputed every step as an FP32 dot product of n terms):
  B = gamma_{n+1} (|bt| + |At| |x_k|), gamma_j = j u / (1 - j u).
* GRAM path (r_{k+1} = fl(r_k - alpha_k G~[:, i_k]), r_{i_k} := 0, x updated
  by FMA, FP64 recomputation every K steps): with G~ the split-BF16 Gram
  matrix, |G~ - G| <= c_G (|At| |At|^T) entrywise, and P = |At| |x|,
    refresh step:  B = u |r_k| + 2 gamma64 P_k       (FP64 dot, rounded once)
    other steps:   B_{k+1,j} = B_{k,j} + |alpha_k| c_G S_j
                               + u (|r_{k+1,j}| + B_{k,j} + |alpha_k| c_G S_j)
                               + u P_{k+1,j}     (rounding of the x update)
                   B_{k+1,i_k} = |r_{k+1,i_k}|   (the GPU holds 0 there)
  with S = |At| |At_{i_k}|^T and |alpha_k| <= (|r_{k,i_k}| + B_{k,i_k}) /
  ||At_{i_k}||^2 (1 + 4u).  The bound grows with the drift since the last
  refresh, which is what it has to cover.
* UPDATE path (the residual-update form of Remark 1: r_{k+1} = r_k - alpha_k
  fl(At At_{i_k}^T), r_{i_k} := 0, recomputed as bt - At x in the working
  precision at step 0 and every K steps): the GRAM recursion with c_G
  replaced by gamma_n, the error of each dot product At_j . At_{i_k}, and the
  GEMV bound at the recomputation steps.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

U32 = 2.0 ** -24
U64 = 2.0 ** -53

# One line per check, printed in the terminal summary (conftest.py).
REPORT: list[str] = []


def split_bf16_coeff(n: int) -> float:
    """c_G: split-BF16 product with FP32 accumulation on the tensor cores.
    Dropping lo*lo and rounding lo cost 2^-14 relative per product; the
    accumulation rounds once per K = 16 instruction, M = 3 k_pad / 16 of them
    (k_pad = 64 ceil(n / 64)), each at most 2^-23 relative."""
    M = 3 * ((n + 63) // 64 * 64) // 16
    return 2.0 ** -14 + (M + 16) * 2.0 ** -23


@dataclass
class StepReport:
    name: str
    steps: int = 0             # steps checked by the replay (selection + projection)
    forced: int = 0            # steps where the bound proves i_k is the unique maximiser
    oracle_compared: int = 0   # steps where the oracle selected from the GPU's x_k
    oracle_equal: int = 0      # ... and picked the GPU's i_k
    oracle_forced: int = 0     # ... of which the oracle's pick was forced (must be equal)
    prefix: int | None = None  # common prefix with the oracle's own trajectory
    notes: list = field(default_factory=list)

    def line(self) -> str:
        s = (f"{self.name}: replayed {self.steps} steps, {self.forced} forced by the bound; "
             f"oracle from the GPU iterate at {self.oracle_compared} steps, "
             f"{self.oracle_equal} equal ({self.oracle_forced} forced)")
        if self.prefix is not None:
            s += f"; common prefix with the oracle's trajectory {self.prefix} steps"
        return s


def _keys(R, B, N, valid, u):
    hi = np.where(valid, (np.abs(R) + B) ** 2 / np.where(valid, N, 1) * (1 + 8 * u), -1.0)
    lo = np.where(valid, np.maximum(np.abs(R) - B, 0) ** 2 / np.where(valid, N, 1) * (1 - 8 * u),
                  -1.0)
    return hi, lo


def replay(At, bt, X, ik, steps, path="gemv", refresh=0, u=U32, name="", oracle=None,
           oracle_steps=None, nthreads=8, block=256) -> StepReport:
    """Check `steps` GPU steps (needs X[0..steps] and ik[0..steps-1]).

    path: "gemv" (residual recomputed every step), "gram" (updated with
    the split-BF16 Gram matrix, FP64 recomputation at steps 0, K, 2K, ... for
    refresh = K > 0, at step 0 only for refresh = 0 -- the batched loop with
    x0 = 0 starts from r = bt exactly, which the refresh formula covers) or
    "update" (updated with dot products against the chosen row, recomputed in
    the working precision at steps 0, K, 2K, ...).
    oracle: the oracle module, to run its own selection from each x_k at the
    steps `oracle_steps` (default: all).  The residuals of a block of steps
    are formed with one matrix product."""
    A = np.asarray(At, np.float64)
    b = np.asarray(bt, np.float64)
    d, n = A.shape
    N = np.sum(A * A, axis=1)
    valid = N > 0
    absA = np.abs(A)
    Xd = np.asarray(X[:steps + 1], np.float64)
    ik = np.asarray(ik[:steps], np.int64)
    rep = StepReport(name or path)
    g = (n + 1) * u / (1 - (n + 1) * u)
    g64 = (n + 2) * U64
    cg = split_bf16_coeff(n) if path == "gram" else n * u / (1 - n * u)
    B = None
    for k0 in range(0, steps, block):
        k1 = min(steps, k0 + block)
        Rb = b[:, None] - A @ Xd[k0:k1 + 1].T          # r at x_k0 .. x_k1
        Pb = absA @ np.abs(Xd[k0:k1 + 1]).T
        Sb = absA @ absA[ik[k0:k1]].T if path in ("gram", "update") else None
        for k in range(k0, k1):
            q = k - k0
            x, x1 = Xd[k], Xd[k + 1]
            R, P = Rb[:, q], Pb[:, q]
            fresh = k == 0 or (refresh > 0 and k % refresh == 0)
            if path == "gemv" or (path == "update" and fresh):
                B = g * (np.abs(b) + P)
            elif fresh:
                B = u * np.abs(R) + 2 * g64 * P
            # (gram, update: B carried over from the previous step otherwise)
            j = int(ik[k])
            assert 0 <= j < d and valid[j], (name, k, j)
            hi, lo = _keys(R, B, N, valid, u)
            others = np.delete(hi, j)
            assert hi[j] >= lo.max(), (name, "selection", k, j, hi[j], lo.max())
            if others.size == 0 or lo[j] > others.max():
                rep.forced += 1
            alpha = R[j] / N[j]
            da = B[j] / N[j] + 4 * u * abs(alpha)
            err = np.abs((x1 - x) - alpha * A[j])
            assert np.all(err <= da * absA[j] + 2 * u * (np.abs(x) + np.abs(x1))), \
                (name, "projection", k)
            rep.steps += 1
            if oracle is not None and (oracle_steps is None or k in oracle_steps):
                ref = oracle.mwrk(A, b, x0=x, tol=0.0, max_iter=1, log_len=1, nthreads=nthreads)
                jo = int(ref.ik[0])
                rep.oracle_compared += 1
                others_o = np.delete(hi, jo)
                forced_o = bool(others_o.size == 0 or lo[jo] > others_o.max())
                rep.oracle_forced += int(forced_o)
                if jo == j:
                    rep.oracle_equal += 1
                else:
                    # a different pick is allowed only where both rows are admissible
                    assert not forced_o and hi[jo] >= lo.max(), (name, "oracle pick", k, j, jo)
            if path in ("gram", "update"):
                R1, P1 = Rb[:, q + 1], Pb[:, q + 1]
                amax = (abs(R[j]) + B[j]) / N[j] * (1 + 4 * u)
                drift = amax * cg * Sb[:, q]
                Bn = B + drift + u * (np.abs(R1) + B + drift) + u * P1
                Bn[j] = abs(R1[j]) * (1 + u)
                B = Bn
    return rep


def trajectory_prefix(ik_gpu, ref, tau):
    """Common prefix of the GPU's i_k with the oracle's own trajectory, and
    k_tau, the first step whose oracle selection gap (t1 - t2) / t1 is below
    tau: two rows that close may be ordered either way by the rounding of the
    two sides, after which the trajectories part.  Asserts the sequences
    agree at least up to min(1000, k_tau)."""
    gap = ref.gap
    k_tau = int(np.argmax(gap < tau)) if np.any(gap < tau) else len(gap)
    L = min(len(ik_gpu), len(ref.ik))
    diff = np.flatnonzero(np.asarray(ik_gpu[:L]) != np.asarray(ref.ik[:L]))
    K = int(diff[0]) if len(diff) else L
    need = min(1000, k_tau, L)
    assert K >= need, (K, need, k_tau)
    return K, k_tau


def record(rep: StepReport):
    REPORT.append(rep.line())
    return rep
