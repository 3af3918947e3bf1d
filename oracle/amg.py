"""Classical (Ruge-Stueben) AMG coarsening of Sec. 3.1 (oracle; test infrastructure).

Sec. 3.2 applies the classical AMG setup to the diffusion-type operator
G_L = L^T D^2 L of eq. (normal) and uses its interpolation operators P_k for
the one-sided hierarchies A_{k+1} = A_k P_k, M_{k+1} = M_k P_k.  The setup,
for a matrix K:

  * strong connections: j != i is a strong connection of row i unless
    -k_ij <= theta * max_{m != i} (-k_im), theta = 0.25;
  * first pass: a greedy maximal independent set of the strength graph.
    Every point starts with the measure "number of its strong connections";
    repeatedly the unsorted point of largest measure becomes a C point, its
    unsorted strong neighbours become F points, and the unsorted strong
    neighbours of each new F point have their measure raised by one;
  * second pass: F points move to C where interpolation would otherwise
    lack a common C point (below);
  * interpolation: C points inject; an F point i interpolates from the set
    C_i of its strong C connections with the weights

        w_ij = -(k_ij + sum_{m in F_i^s} k_im k_mj / sum_{l in C_i} k_ml)
                / (k_ii + sum_{m in F_i^w} k_im),

    F_i^s its strong F connections and F_i^w the rest of its neighbours;
  * coarse operators K_{k+1} = P_k^T K_k P_k (Galerkin).

Readings taken where the paper names the steps, not these details:
  * "strong connections of i" are the j in S_i = {j : -k_ij > theta max};
    "its strong neighbours" of a new C point i are the unsorted points that
    depend strongly on i (i in S_j), as Ruge and Stueben define the
    transpose set S_i^T, and the measure is |S_i^T|;
  * a threshold tie is weak: -k_ij must exceed theta * max * (1 + 1e-10),
    so values that are equal in exact arithmetic are decided the same way
    whatever the rounding order of the Galerkin products that made them;
  * ties of the measure go to the smallest index; only the increment the
    paper names is applied (no decrement of the new C point's own strong
    connections);
  * second pass, F points in increasing index: for F point i with
    C_i = S_i intersect C, each strong F connection j (increasing index)
    that has no strong connection into C_i is tentatively made a C point
    (and joins C_i); if a second such j appears, i itself becomes a C point
    and the tentative point stays F; a tentative point that survives the
    scan becomes C;
  * the coarse points are numbered in increasing fine index;
  * a strong F neighbour m whose sum over C_i is exactly zero is counted
    with F_i^w (lumped into the diagonal);
  * coarsening stops at `max_levels` levels, when a level has at most
    `max_coarse` points, or when a pass keeps every point.

Parallel replacement of the two passes (method="pmis"; De Sterck, Yang and
Heys' PMIS, 2006): every point's measure is |S_i^T| plus a uniform random
number in [0, 1); a point with no strong connection in either direction is
F (a reading: PMIS makes every point nothing depends on F, which can leave
an F point with no C point to interpolate from); then, in rounds, every unsorted point whose (measure, index) exceeds that of each
unsorted point it is strongly connected to in either direction becomes C,
and every unsorted point with a strong connection to a C point becomes F.
The random numbers are SplitMix64 (Steele, Lea and Flood 2014) outputs of
the stream seeded with PMIS_SEED + level, each mapped to (z >> 11) 2^-53.
Interpolation is the paper's formula as above; its lumping rule covers the
strong F-F pairs without a common C point that PMIS leaves.

Every step is a plain loop over rows in the order stated; scipy is used for
the sparse products only.
"""
from __future__ import annotations

import heapq

import numpy as np
import scipy.sparse as sp

THETA = 0.25
TIE_REL = 1e-10
C_PT, F_PT = 1, 0
PMIS_SEED = 2306
_M64 = (1 << 64) - 1


def _rows(K):
    K = sp.csr_matrix(K, dtype=np.float64)
    K.sort_indices()
    return K


def strength(K, theta=THETA):
    """S[i]: increasing list of the strong connections of row i."""
    K = _rows(K)
    S = []
    for i in range(K.shape[0]):
        cols = K.indices[K.indptr[i]:K.indptr[i + 1]]
        vals = K.data[K.indptr[i]:K.indptr[i + 1]]
        off = [(j, -v) for j, v in zip(cols, vals) if j != i]
        mx = max((nv for _, nv in off), default=0.0)
        thr = theta * mx * (1.0 + TIE_REL)
        S.append([int(j) for j, nv in off if mx > 0.0 and nv > thr])
    return S


def transpose_sets(S, n):
    ST = [[] for _ in range(n)]
    for i in range(n):
        for j in S[i]:
            ST[j].append(i)
    return ST


def first_pass(S, n):
    """Greedy C/F split (C_PT / F_PT per point)."""
    ST = transpose_sets(S, n)
    measure = [len(ST[i]) for i in range(n)]
    cf = [None] * n
    heap = [(-measure[i], i) for i in range(n)]
    heapq.heapify(heap)
    left = n
    while left:
        negm, i = heapq.heappop(heap)
        if cf[i] is not None or -negm != measure[i]:
            continue                                  # sorted, or a stale entry
        cf[i] = C_PT
        left -= 1
        new_f = [j for j in ST[i] if cf[j] is None]
        for j in new_f:
            cf[j] = F_PT
            left -= 1
        for j in new_f:
            for k in S[j]:
                if cf[k] is None:
                    measure[k] += 1
                    heapq.heappush(heap, (-measure[k], k))
    return np.array(cf, dtype=np.int8)


def second_pass(S, cf):
    cf = np.array(cf, dtype=np.int8)
    n = cf.size
    for i in range(n):
        if cf[i] != F_PT:
            continue
        Ci = {j for j in S[i] if cf[j] == C_PT}
        tentative = None
        for j in S[i]:
            if cf[j] != F_PT:
                continue
            if any(l in Ci for l in S[j]):
                continue
            if tentative is None:
                tentative = j
                Ci.add(j)
            else:
                cf[i] = C_PT
                tentative = None
                break
        if tentative is not None:
            cf[tentative] = C_PT
    return cf


def split(K, theta=THETA):
    """C/F split of the two passes, and the strength sets."""
    S = strength(K, theta)
    cf = first_pass(S, len(S))
    return second_pass(S, cf), S


def splitmix64_uniform(seed, n):
    """n uniforms in [0, 1) from the SplitMix64 stream seeded with `seed`."""
    out = np.empty(n)
    state = seed & _M64
    for i in range(n):
        state = (state + 0x9E3779B97F4A7C15) & _M64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        z ^= z >> 31
        out[i] = (z >> 11) * 2.0 ** -53
    return out


def pmis_split(S, n, rand):
    """PMIS C/F split of the strength sets S with the random numbers rand."""
    ST = transpose_sets(S, n)
    w = [len(ST[i]) + float(rand[i]) for i in range(n)]
    nbr = [sorted(set(S[i]) | set(ST[i])) for i in range(n)]
    U = -1
    cf = [U] * n
    for i in range(n):
        if not ST[i] and not S[i]:
            cf[i] = F_PT
    while U in cf:
        new_c = [i for i in range(n) if cf[i] == U and
                 all((w[i], i) > (w[j], j) for j in nbr[i] if cf[j] == U)]
        for i in new_c:
            cf[i] = C_PT
        for i in range(n):
            if cf[i] == U and any(cf[j] == C_PT for j in S[i]):
                cf[i] = F_PT
    return np.array(cf, dtype=np.int8)


def interpolation(K, S, cf) -> sp.csr_matrix:
    """P (n x n_c) of the paper's interpolation formula."""
    K = _rows(K)
    n = K.shape[0]
    cidx = -np.ones(n, dtype=np.int64)
    cpts = np.flatnonzero(cf == C_PT)
    cidx[cpts] = np.arange(cpts.size)
    row = [dict(zip(K.indices[K.indptr[i]:K.indptr[i + 1]].tolist(),
                    K.data[K.indptr[i]:K.indptr[i + 1]].tolist())) for i in range(n)]
    rows, cols, vals = [], [], []
    for i in range(n):
        if cf[i] == C_PT:
            rows.append(i); cols.append(cidx[i]); vals.append(1.0)
            continue
        Si = set(S[i])
        Ci = [j for j in S[i] if cf[j] == C_PT]
        Fs = []
        den = row[i].get(i, 0.0)
        for m, kim in sorted(row[i].items()):
            if m == i or (m in Si and cf[m] == C_PT):
                continue
            if m in Si:
                tot = sum(row[m].get(l, 0.0) for l in Ci)
                if tot != 0.0:
                    Fs.append((m, kim, tot))
                    continue
            den += kim                                    # F_i^w (and weak C points)
        for j in Ci:
            num = row[i].get(j, 0.0)
            for m, kim, tot in Fs:
                num += kim * row[m].get(j, 0.0) / tot
            rows.append(i); cols.append(cidx[j]); vals.append(-num / den)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, cpts.size))


def hierarchy(K0, max_levels=20, max_coarse=256, theta=THETA, method="rs"):
    """Operators K_k, interpolations P_k (level k+1 -> k) and splits;
    method "rs" (the paper's two passes) or "pmis"."""
    Ks, Ps, cfs = [_rows(K0)], [], []
    while len(Ks) < max_levels and Ks[-1].shape[0] > max_coarse:
        if method == "pmis":
            S = strength(Ks[-1], theta)
            n = len(S)
            cf = pmis_split(S, n, splitmix64_uniform(PMIS_SEED + len(Ks) - 1, n))
        else:
            cf, S = split(Ks[-1], theta)
        if cf.sum() in (0, cf.size):
            break
        P = interpolation(Ks[-1], S, cf)
        Ps.append(P)
        cfs.append(cf)
        Ks.append(_rows(P.T @ Ks[-1] @ P))
    return Ks, Ps, cfs
