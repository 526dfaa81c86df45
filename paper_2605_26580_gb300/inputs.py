"""Seeded synthetic inputs: regular GF(2^m) LDPC codes, interleavers, codewords, y.

This module is shared by the test suite, the benchmark and the CPU oracle's
callers as the single source of inputs.  It holds none of the decoder's
arithmetic: it builds parity-check matrices (appendix "Q-ary LDPC code",
paragraph "Construction of H": random nonzero positions, i.i.d. coefficients
uniform on F_Q^x), an encoder (Gaussian elimination over GF(2^m), used only to
draw uniform codewords) and the K-user PAM-sum channel output

    y_t = sum_k (2 c_{k, pi_k^{-1}(t)} - (Q-1)) + w_t,   w_t ~ N(0, sigma2),
    sigma2 = E_s 10^(-SNR/10),  E_s = (Q^2 - 1)/3 (mean energy of a uniform level).

Random numbers come from NumPy's PCG64 with explicit seeds.  Its GF(2^m)
arithmetic is its own (exp/log tables from the same primitive polynomials the
decoder uses: x^2+x+1, x^4+x+1, x^6+x+1, ...), independent of the oracle's and
of the CUDA library's.
"""
from __future__ import annotations

import math

import numpy as np

PRIM_POLY = {1: 0x3, 2: 0x7, 3: 0xB, 4: 0x13, 5: 0x25, 6: 0x43, 7: 0x89, 8: 0x11D}


def code_seed(n: int, q: int) -> int:
    """Default seed of the (n, q) code: 2605e6 + q*1e4 + n."""
    return 2605 * 10**6 + q * 10**4 + n


def log2_exact(q: int) -> int:
    m = int(q).bit_length() - 1
    if q < 2 or (1 << m) != q or m > 8:
        raise ValueError("q must be 2^m with 1 <= m <= 8, got %r" % (q,))
    return m


class _GF:
    """GF(2^m) by exp/log tables (for the encoder only)."""

    def __init__(self, m: int):
        self.m, self.q = m, 1 << m
        q = self.q
        exp = np.zeros(2 * q, dtype=np.int64)
        log = np.zeros(q, dtype=np.int64)
        x = 1
        for i in range(q - 1):
            exp[i] = x
            log[x] = i
            x <<= 1
            if x & q:
                x ^= PRIM_POLY[m]
        for i in range(q - 1, 2 * q):
            exp[i] = exp[i - (q - 1)]
        a = np.arange(q)[:, None]
        b = np.arange(q)[None, :]
        mul = exp[(log[a] + log[b]) % (q - 1)]
        mul[(a == 0) | (b == 0)] = 0
        self.mul = mul.astype(np.int64)
        self.inv = np.zeros(q, dtype=np.int64)
        for v in range(1, q):
            self.inv[v] = exp[(q - 1 - log[v]) % (q - 1)]


def _four_cycle_edges(chk_var: np.ndarray, P: int, dc: int) -> np.ndarray:
    """Edges that sit on a double edge or a 4-cycle of the Tanner graph."""
    rows = chk_var.reshape(P, dc)
    bad = np.zeros(P * dc, dtype=bool)
    for j in range(P):
        vals, counts = np.unique(rows[j], return_counts=True)
        for v in vals[counts > 1]:
            bad[j * dc + np.nonzero(rows[j] == v)[0]] = True
    var_checks: dict[int, list[int]] = {}
    for e, v in enumerate(chk_var.tolist()):
        var_checks.setdefault(v, []).append(e // dc)
    seen: dict[tuple[int, int], int] = {}
    for v, cs in var_checks.items():
        cs = sorted(set(cs))
        for a in range(len(cs)):
            for b in range(a + 1, len(cs)):
                key = (cs[a], cs[b])
                if key in seen:
                    for vv in (v, seen[key]):
                        for j in key:
                            bad[j * dc + np.nonzero(rows[j] == vv)[0]] = True
                else:
                    seen[key] = v
    return np.nonzero(bad)[0]


def make_code(n: int, q: int, dv: int = 2, dc: int = 4, seed: int | None = None) -> dict:
    """Regular (dv, dc) GF(q) LDPC code with no double edges and no 4-cycles.

    Socket model: the n*dv variable sockets are placed on the P*dc check sockets
    by a seeded random permutation (check-major: check j owns edges j*dc..j*dc+dc-1);
    offending edges are then swapped with random edges until the graph has no
    repeated variable in a check and no two variables sharing two checks.
    Coefficients are i.i.d. uniform on {1, ..., q-1}.
    """
    m = log2_exact(q)
    if (n * dv) % dc:
        raise ValueError("n*dv must be a multiple of dc")
    P = n * dv // dc
    rng = np.random.Generator(np.random.PCG64(code_seed(n, q) if seed is None else seed))
    sockets = np.repeat(np.arange(n, dtype=np.int64), dv)
    chk_var = sockets[rng.permutation(n * dv)]
    for _ in range(100000):
        bad = _four_cycle_edges(chk_var, P, dc)
        if bad.size == 0:
            break
        e1 = int(rng.choice(bad))
        e2 = int(rng.integers(0, n * dv))
        chk_var[e1], chk_var[e2] = chk_var[e2], chk_var[e1]
    else:
        raise RuntimeError("could not remove 4-cycles")
    chk_coef = rng.integers(1, q, size=P * dc)
    code = {"n": n, "P": P, "q": q, "m": m, "dv": dv, "dc": dc,
            "chk_var": chk_var.astype(np.int32), "chk_coef": chk_coef.astype(np.uint8)}
    code.update(_encoder(code))
    return code


def make_irregular_code(n: int, q: int, profile: dict, dc: int, seed: int | None = None) -> dict:
    """GF(q) LDPC code with an irregular variable-degree profile and check degree dc.

    profile maps a variable degree to the fraction of variables that have it
    (e.g. {2: 0.5, 3: 0.3, 4: 0.2}).  The per-degree counts are the rounded
    fractions, then variables move one degree down (from the largest degree
    present) until the edge count is a multiple of dc; degrees are assigned to
    variables by a seeded shuffle.  The sockets are then placed and repaired as in
    make_code (no double edges, no 4-cycles); coefficients i.i.d. uniform on
    {1, ..., q-1} (appendix "Construction of H": a sampled sparse support with
    i.i.d. nonzero coefficients).  code["dv"] is the largest degree.
    """
    m = log2_exact(q)
    rng = np.random.Generator(np.random.PCG64((code_seed(n, q) + 29) if seed is None else seed))
    degs = sorted(profile)
    counts = {d: int(round(profile[d] * n)) for d in degs}
    counts[degs[0]] += n - sum(counts.values())
    total = sum(d * c for d, c in counts.items())
    while total % dc:
        top = max(d for d in degs if counts[d] > 0 and d > 1)
        counts[top] -= 1
        counts[top - 1] = counts.get(top - 1, 0) + 1
        total -= 1
    deg = np.concatenate([np.full(c, d, dtype=np.int64) for d, c in sorted(counts.items()) if c > 0])
    deg = deg[rng.permutation(n)]
    P = int(deg.sum()) // dc
    sockets = np.repeat(np.arange(n, dtype=np.int64), deg)
    chk_var = sockets[rng.permutation(sockets.size)]
    for _ in range(100000):
        bad = _four_cycle_edges(chk_var, P, dc)
        if bad.size == 0:
            break
        e1 = int(rng.choice(bad))
        e2 = int(rng.integers(0, sockets.size))
        chk_var[e1], chk_var[e2] = chk_var[e2], chk_var[e1]
    else:
        raise RuntimeError("could not remove 4-cycles")
    chk_coef = rng.integers(1, q, size=P * dc)
    code = {"n": n, "P": P, "q": q, "m": m, "dv": int(deg.max()), "dc": dc,
            "chk_var": chk_var.astype(np.int32), "chk_coef": chk_coef.astype(np.uint8), "var_deg": deg.astype(np.int32)}
    code.update(_encoder(code))
    return code


def make_peg_code(n: int, q: int, dv: int = 2, dc: int = 3, seed: int | None = None) -> dict:
    """Regular (dv, dc) GF(q) LDPC code by progressive edge growth.

    Variables are placed one at a time.  A variable's first edge goes to a check
    of the lowest current degree; each further edge goes to a check as far as
    possible from the variable in the graph built so far (unreachable checks
    first, else those at the largest breadth-first depth), again of the lowest
    current degree.  Only checks below degree dc are candidates, so the code is
    check-regular; remaining ties are broken by a seeded random draw.
    Coefficients are i.i.d. uniform on {1, ..., q-1}.
    """
    m = log2_exact(q)
    if (n * dv) % dc:
        raise ValueError("n*dv must be a multiple of dc")
    P = n * dv // dc
    rng = np.random.Generator(np.random.PCG64((code_seed(n, q) + 11) if seed is None else seed))
    var_chk = [[] for _ in range(n)]
    chk_vars = [[] for _ in range(P)]
    for v in range(n):
        for k in range(dv):
            open_ = [c for c in range(P) if len(chk_vars[c]) < dc and c not in var_chk[v]]
            if k == 0:
                cand = open_
            else:
                # breadth-first depths of the checks reachable from v
                depth = {}
                frontier = list(var_chk[v])
                for c in frontier:
                    depth[c] = 0
                seen_v = {v}
                d = 0
                while frontier:
                    nxt = []
                    for c in frontier:
                        for u in chk_vars[c]:
                            if u in seen_v:
                                continue
                            seen_v.add(u)
                            for c2 in var_chk[u]:
                                if c2 not in depth:
                                    depth[c2] = d + 1
                                    nxt.append(c2)
                    frontier = nxt
                    d += 1
                far = [c for c in open_ if c not in depth]
                if not far:
                    best = max(depth[c] for c in open_)
                    far = [c for c in open_ if depth[c] == best]
                cand = far
            low = min(len(chk_vars[c]) for c in cand)
            cand = [c for c in cand if len(chk_vars[c]) == low]
            c = int(cand[int(rng.integers(0, len(cand)))])
            var_chk[v].append(c)
            chk_vars[c].append(v)
    chk_var = np.array([v for c in range(P) for v in chk_vars[c]], dtype=np.int32)
    chk_coef = rng.integers(1, q, size=P * dc).astype(np.uint8)
    code = {"n": n, "P": P, "q": q, "m": m, "dv": dv, "dc": dc, "chk_var": chk_var, "chk_coef": chk_coef}
    code.update(_encoder(code))
    return code


def girth(code: dict) -> int:
    """Length of the shortest cycle of the Tanner graph (breadth-first from every
    variable; 0 if the graph has no cycle)."""
    n, P, dc = code["n"], code["P"], code["dc"]
    cv = np.asarray(code["chk_var"]).reshape(P, dc)
    var_chk = [[] for _ in range(n)]
    for j in range(P):
        for v in cv[j]:
            var_chk[int(v)].append(j)
    best = 0
    for s in range(n):
        # nodes: variables as ("v", i), checks as ("c", j); BFS with parent tracking
        dist = {("v", s): 0}
        parent = {("v", s): None}
        queue = [("v", s)]
        qi = 0
        while qi < len(queue):
            node = queue[qi]
            qi += 1
            kind, idx = node
            nbrs = [("c", j) for j in var_chk[idx]] if kind == "v" else [("v", int(u)) for u in cv[idx]]
            for nb in nbrs:
                if nb == parent[node]:
                    continue
                if nb in dist:
                    cyc = dist[node] + dist[nb] + 1
                    if best == 0 or cyc < best:
                        best = cyc
                else:
                    dist[nb] = dist[node] + 1
                    parent[nb] = node
                    queue.append(nb)
    return best


def code_from_edges(n: int, q: int, dc: int, chk_var, chk_coef) -> dict:
    """Wrap an explicit check-major edge list (any variable degrees)."""
    chk_var = np.asarray(chk_var, dtype=np.int32).reshape(-1)
    chk_coef = np.asarray(chk_coef, dtype=np.uint8).reshape(-1)
    if chk_var.size % dc:
        raise ValueError("edge count must be a multiple of dc")
    deg = np.bincount(chk_var, minlength=n)
    code = {"n": n, "P": chk_var.size // dc, "q": q, "m": log2_exact(q), "dv": int(deg.max()), "dc": dc,
            "chk_var": chk_var, "chk_coef": chk_coef}
    code.update(_encoder(code))
    return code


def _encoder(code: dict) -> dict:
    """Systematic encoder from Gaussian elimination of H over GF(q).

    Returns the information positions (non-pivot columns), rank(H) and a binary
    generator that maps information bits to codeword bits (multiplication by a
    fixed field element is GF(2)-linear, so encoding is a 0/1 matrix product).
    """
    n, P, q, m, dc = code["n"], code["P"], code["q"], code["m"], code["dc"]
    gf = _GF(m)
    H = np.zeros((P, n), dtype=np.int64)
    for e in range(P * dc):
        H[e // dc, int(code["chk_var"][e])] = int(code["chk_coef"][e])
    pivots = []
    r = 0
    for c in range(n):
        if r == P:
            break
        nz = np.nonzero(H[r:, c])[0]
        if nz.size == 0:
            continue
        p = r + int(nz[0])
        if p != r:
            H[[r, p]] = H[[p, r]]
        H[r] = gf.mul[gf.inv[H[r, c]], H[r]]
        rows = np.nonzero(H[:, c])[0]
        rows = rows[rows != r]
        if rows.size:
            H[rows] ^= gf.mul[H[rows, c][:, None], H[r][None, :]]
        pivots.append(c)
        r += 1
    rank = r
    piv = np.array(pivots, dtype=np.int64)
    info = np.array(sorted(set(range(n)) - set(pivots)), dtype=np.int64)
    k = info.size
    # generator over GF(2): bit b of info symbol f -> bits of every codeword symbol
    G = np.zeros((k * m, n * m), dtype=np.float32)
    for fi, col in enumerate(info):
        for b in range(m):
            G[fi * m + b, col * m + b] = 1.0
    for row in range(rank):
        for fi, col in enumerate(info):
            h = int(H[row, col])
            if h == 0:
                continue
            for b in range(m):
                prod = int(gf.mul[h, 1 << b])
                for b2 in range(m):
                    if (prod >> b2) & 1:
                        G[fi * m + b, piv[row] * m + b2] = 1.0
    return {"rank": rank, "k": k, "info_pos": info.astype(np.int32), "gen_bits": G}


def encode(code: dict, info: np.ndarray, device=None) -> np.ndarray:
    """Codewords [..., n] (uint8) for information symbols [..., k].

    The 0/1 matrix product is exact in float32 (sums < 2^24) on any device;
    device = a torch device runs it there (the result is identical)."""
    m, n, k = code["m"], code["n"], code["k"]
    shape = info.shape[:-1]
    flat = np.asarray(info, dtype=np.int64).reshape(-1, k)
    bits = ((flat[:, :, None] >> np.arange(m)[None, None, :]) & 1).astype(np.float32).reshape(-1, k * m)
    out = np.empty((flat.shape[0], n), dtype=np.uint8)
    weights = (1 << np.arange(m)).astype(np.int64)
    G = code["gen_bits"]
    step = 16384
    if device is not None:
        import torch
        Gd = torch.from_numpy(G).to(device)
        wd = torch.from_numpy(weights).to(device)
        for s in range(0, flat.shape[0], step):
            cb = (torch.from_numpy(bits[s:s + step]).to(device) @ Gd).to(torch.int64) & 1
            out[s:s + step] = (cb.reshape(-1, n, m) * wd).sum(-1).to(torch.uint8).cpu().numpy()
        return out.reshape(*shape, n)
    for s in range(0, flat.shape[0], step):
        cb = (bits[s:s + step] @ G).astype(np.int64) & 1   # exact: 0/1 sums < 2^24
        out[s:s + step] = (cb.reshape(-1, n, m) * weights).sum(-1).astype(np.uint8)
    return out.reshape(*shape, n)


def make_interleavers(n: int, K: int, seed: int, interleave: bool = True) -> np.ndarray:
    """pi[k, i] = channel use of user k's symbol i; pi_0 = identity."""
    pi = np.tile(np.arange(n, dtype=np.int32), (K, 1))
    if interleave:
        rng = np.random.Generator(np.random.PCG64(seed))
        for k in range(1, K):
            pi[k] = rng.permutation(n).astype(np.int32)
    return pi


def es(q: int) -> float:
    """Mean energy of the uniform PAM levels 2a-(q-1): (q^2-1)/3."""
    return (q * q - 1) / 3.0


def sigma2_from_snr(q: int, snr_db: float) -> float:
    return es(q) * 10.0 ** (-snr_db / 10.0)


def channel_output(q: int, c: np.ndarray, perm: np.ndarray, snr_db, seed: int,
                   noiseless: bool = False) -> tuple[np.ndarray, float]:
    """y [F, n] float32 of codewords c [F, K, n] through the PAM-sum channel.
    snr_db: a scalar or one value per frame (then sigma2 is returned per frame)."""
    F, K, n = c.shape
    sigma2 = sigma2_from_snr(q, np.asarray(snr_db, dtype=np.float64)) if np.ndim(snr_db) else sigma2_from_snr(q, snr_db)
    y = np.zeros((F, n), dtype=np.float64)
    for k in range(K):
        y[:, perm[k]] += 2.0 * c[:, k, :].astype(np.float64) - (q - 1)
    if not noiseless:
        rng = np.random.Generator(np.random.PCG64(seed))
        scale = np.sqrt(sigma2)[:, None] if np.ndim(sigma2) else math.sqrt(sigma2)
        y += rng.standard_normal((F, n)) * scale
    return y.astype(np.float32), sigma2


def make_frames(code: dict, K: int, snr_db: float, F: int, seed: int, interleave: bool = True,
                noiseless: bool = False, perm_seed: int | None = None, device=None) -> dict:
    """F frames of K users: uniform info symbols, codewords, channel output y (float32).

    Streams: info symbols from PCG64(seed), interleavers from PCG64(perm_seed or
    seed), noise from PCG64(seed + 1)."""
    q, n = code["q"], code["n"]
    rng = np.random.Generator(np.random.PCG64(seed))
    info = rng.integers(0, q, size=(F, K, code["k"]), dtype=np.int64)
    c = encode(code, info, device)                           # [F, K, n]
    pi = make_interleavers(n, K, seed if perm_seed is None else perm_seed, interleave)
    y, sigma2 = channel_output(q, c, pi, snr_db, seed + 1, noiseless)
    return {"c": c, "y": y, "sigma2": sigma2, "perm": pi, "snr_db": snr_db, "K": K,
            "info": info.astype(np.int32)}


def random_log_messages(rng: np.random.Generator, shape, q: int, spread: float = 8.0,
                        log_floor: float = math.log(1e-12)) -> np.ndarray:
    """Random max-normalised log-messages [..., q] for single-step tests: Gaussian
    logits scaled by `spread`, shifted to max 0 and clipped at log_floor."""
    x = rng.standard_normal(tuple(shape) + (q,)) * spread
    x -= x.max(axis=-1, keepdims=True)
    return np.maximum(x, log_floor)


# ---------------------------------------------------------------------------
# Evidence interface (the paper's URA slot model; appendix "Unsourced random
# access", appendix "Simulation pipeline and channel model")
# ---------------------------------------------------------------------------

def ura_rows(L: int, q: int, ns: int, seed: int) -> np.ndarray:
    """Partial-DFT row indices [L, ns] (int32): per slot, ns distinct rows of the
    q x q DFT drawn uniformly from PCG64(seed) (appendix "Sensing-matrix
    construction"; one dictionary per slot, fixed for all frames)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.stack([rng.choice(q, size=ns, replace=False) for _ in range(L)]).astype(np.int32)


def ura_psym(code: dict, eb_db: float) -> float:
    """Transmit power per symbol P_sym = B 10^(Eb/10) / L with B = log2(q) k info
    bits (appendix "Simulation constants")."""
    B = code["m"] * code["k"]
    return B * 10.0 ** (eb_db / 10.0) / code["n"]


def ura_detector_params(K: int, q: int, psym: float) -> dict:
    """Detector hyper-parameters and the SIC cancellation weight, as read here
    (the paper leaves them open): rho_BG = K / q (about K of q signatures
    active per slot), sigma_u^2 = P_sym (power of one unit-amplitude signature
    at the transmit scale), cancel_log = -log q (after a row is decoded, a
    later row uses the same symbol in that slot only by collision, probability
    1/q under uniform symbols)."""
    return {"rho": K / q, "su2": float(psym), "cancel_log": -math.log(q)}


def make_ura_frames(code: dict, K: int, eb_db: float, F: int, seed: int, ns: int = 24,
                    rows_seed: int | None = None, noiseless: bool = False) -> dict:
    """F frames of the URA slot model: K uniform messages encoded by the shared
    code (X [F, K, L]), and per slot l the observation

        Y^(l) = sqrt(P_sym) A^(l) U^(l) + eps,   U^(l) = sum_k e_{X[k, l]},
        A^(l) = F_{R_l,:} / sqrt(ns),  F_{k,a} = exp(-2 pi i k a / q),  eps ~ CN(0, I),

    returned as y [F, L, ns, 2] float32 (real, imaginary).  Streams: messages
    from PCG64(seed), noise from PCG64(seed + 1), rows from PCG64(rows_seed or
    the code seed + 7)."""
    q, L = code["q"], code["n"]
    rng = np.random.Generator(np.random.PCG64(seed))
    info = rng.integers(0, q, size=(F, K, code["k"]), dtype=np.int64)
    X = encode(code, info)                                   # [F, K, L]
    rows = ura_rows(L, q, ns, code_seed(L, q) + 7 if rows_seed is None else rows_seed)
    psym = ura_psym(code, eb_db)
    # dictionary columns: A[l, i, a]
    A = np.exp(-2j * np.pi * ((rows[:, :, None].astype(np.int64) * np.arange(q)[None, None, :]) % q) / q)
    A /= math.sqrt(ns)
    Y = np.zeros((F, L, ns), dtype=np.complex128)
    slot = np.arange(L)[None, :]
    for k in range(K):
        Y += A[slot, :, X[:, k, :].astype(np.int64)]         # column X[f, k, l] of slot l: [F, L, ns]
    Y *= math.sqrt(psym)
    if not noiseless:
        nrng = np.random.Generator(np.random.PCG64(seed + 1))
        Y += (nrng.standard_normal((F, L, ns)) + 1j * nrng.standard_normal((F, L, ns))) * math.sqrt(0.5)
    y = np.stack([Y.real, Y.imag], axis=-1).astype(np.float32)
    return {"X": X, "y": y, "rows": rows, "psym": psym, "K": K, "ns": ns, "eb_db": eb_db,
            **ura_detector_params(K, q, psym)}


def match_rows(hat: np.ndarray, X: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Row alignment of eq. (app_ura_hungarian) for small K by enumerating all K!
    permutations: per frame the permutation with the fewest symbol errors.
    hat, X [F, K, L] -> (symbol errors [F], codeword errors [F])."""
    import itertools
    F, K, L = X.shape
    best_sym = np.full(F, K * L + 1, dtype=np.int64)
    best_cw = np.zeros(F, dtype=np.int64)
    for p in itertools.permutations(range(K)):
        diff = hat != X[:, list(p), :]
        sym = diff.sum(axis=(1, 2))
        cw = diff.any(axis=2).sum(axis=1)
        better = sym < best_sym
        best_sym = np.where(better, sym, best_sym)
        best_cw = np.where(better, cw, best_cw)
    return best_sym, best_cw
