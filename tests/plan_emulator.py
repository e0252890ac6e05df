"""Host-side emulation of the library's launch plans (test infrastructure).

Reads a plan through the C ABI's ``bitonic_debug_plan`` (host code only, no
GPU) and executes it with numpy the way the tile kernel defines it: each CTA
holds a tile whose local index L maps to global position g0 ^ G(L); in each
round thread x holds register r at local index T(x) ^ Roff(r >> VB) ^ (r & VEC-1);
steps compare-exchange registers; rounds are joined by a transpose through
an m-bit shared-memory tile.  Used to check the planner's index arithmetic on
the CPU against the oracle before any GPU run.
"""
from __future__ import annotations

import numpy as np

import paper_1506_01446_gb300 as bt

KIND_STEP = 3  # one-step kernel (the launch kinds of bitonic_debug_plan)
debug_plan = bt.debug_plan


def _xor_span(vectors, count_bits):
    """out[v] = XOR of vectors[j] over set bits j of v, v < 2^count_bits."""
    out = np.zeros(1 << count_bits, dtype=np.int64)
    for j in range(count_bits):
        bit = 1 << j
        out[bit:2 * bit] = out[:bit] ^ int(vectors[j])
    return out


def _global_of_local(gvec, m, L):
    g = np.zeros_like(L)
    for j in range(m):
        g ^= np.where((L >> j) & 1, int(gvec[j]), 0)
    return g


def _swz(lv):
    f = (lv >> 3) ^ (lv >> 6) ^ (lv >> 9) ^ (lv >> 12) ^ (lv >> 15)
    return lv ^ (f & 7)


class Stats:
    def __init__(self):
        self.conflicted_quarter_warps = 0
        self.quarter_warps = 0
        self.uncoalesced_rounds = 0
        self.transposes = 0
        self.warp_local_transposes = 0


def _round_local(rd, log_r, log_t, vb):
    """Local index [thread, register] of a round's layout."""
    nreg = log_r - vb
    T = _xor_span(rd["thr_loc"], log_t)                       # [threads]
    Rv = _xor_span(rd["reg_loc"], nreg)                       # [vectors]
    comp = np.arange(1 << vb)
    L = T[:, None, None] ^ Rv[None, :, None] ^ comp[None, None, :]
    return L.reshape(1 << log_t, 1 << log_r)


def _check_banks(Lr, vb, stats):
    """Quarter warps of 16-byte accesses must hit 8 distinct bank groups."""
    threads = Lr.shape[0]
    vec_idx = Lr[:, ::(1 << vb)] >> vb                        # [threads, vectors]
    phys = _swz(vec_idx)
    for q0 in range(0, threads, 8):
        groups = phys[q0:q0 + 8] & 7                          # [8, vectors]
        for v in range(groups.shape[1]):
            stats.quarter_warps += 1
            if len(np.unique(groups[:, v])) != 8:
                stats.conflicted_quarter_warps += 1


def _apply_steps(regs, steps, desc):
    R = regs.shape[-1]
    for code in steps:
        q, flip = code & 15, bool(code & 16)
        i = np.array([r for r in range(R) if not (r >> q) & 1])
        j = (i ^ ((2 << q) - 1)) if flip else (i | (1 << q))
        a, b = regs[..., i], regs[..., j]
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        regs[..., i] = hi if desc else lo
        regs[..., j] = lo if desc else hi


def emulate(keys: np.ndarray, ascending: bool = True, front: int = 0, stats: Stats | None = None,
            key_bytes: int | None = None):
    """Runs the plan of a len(keys) (+front) sort on a copy of keys."""
    keys = np.asarray(keys)
    if key_bytes is None:
        key_bytes = keys.dtype.itemsize
    dt = np.uint32 if key_bytes == 4 else np.uint64
    kmax = np.iinfo(dt).max
    desc = (not ascending) and key_bytes == 4
    n = keys.size
    nv = n + front
    plan = debug_plan(max(nv, 2), key_bytes)
    N, log_r, log_t = plan["N"], plan["log_r"], plan["log_t"]
    vb = 2 if key_bytes == 4 else 1
    m = log_r + log_t if plan["cfg"] >= 0 else 0
    size = max(N, 1 << m)
    front_pad, tail_pad = (kmax, 0) if desc else (0, kmax)
    a = np.full(size, tail_pad, dtype=dt)
    a[:front] = front_pad
    a[front:front + n] = keys
    lo_real, hi_real = front, front + n
    stats = stats or Stats()
    for (kind, p, hi, lo, flip, di, grid) in plan["launches"]:
        if kind == KIND_STEP:
            q = np.arange(N // 2, dtype=np.int64)
            j = hi
            i = ((q >> j) << (j + 1)) | (q & ((1 << j) - 1))
            pr = (i ^ ((2 << j) - 1)) if flip else (i | (1 << j))
            keep = (i >= lo_real) & (pr < hi_real)
            i, pr = i[keep], pr[keep]
            x, y = a[i].copy(), a[pr].copy()
            sw = (x < y) if desc else (y < x)
            a[i[sw]], a[pr[sw]] = y[sw], x[sw]
            continue
        P = plan["descs"][di]
        assert P["m"] == m
        ctas = np.arange(grid, dtype=np.int64)
        g0 = np.zeros(grid, dtype=np.int64)
        rest = ctas.copy()
        for r in range(int(P["nruns"])):
            w = int(P["run_width"][r])
            g0 |= (rest & ((1 << w) - 1)) << int(P["run_shift"][r])
            rest >>= w
        assert np.all(rest == 0), "CTA index does not fit the free bits"
        if P["contiguous"]:
            live = g0 < hi_real
            ctas, g0 = ctas[live], g0[live]
        nr = int(P["nrounds"])
        rounds = P["rounds"][:nr]
        c = int(P["row_log"])
        layouts = [_round_local(rd, log_r, log_t, vb) for rd in rounds]
        for rd, Lr in zip(rounds, layouts):
            assert np.array_equal(np.sort(Lr.ravel()), np.arange(1 << m)), "round layout not a bijection"
            _check_banks(Lr, vb, stats)
            # the planner's precomputed shared-memory slots (byte offsets of
            # 16-byte vectors): thread part XOR register part must equal the
            # swizzle of every vector's local index, times 16
            slot = (_xor_span(rd["thr_sw"], log_t)[:, None]
                    ^ _xor_span(rd["reg_sw"], log_r - vb)[None, :])
            assert np.array_equal(slot, _swz(Lr[:, ::(1 << vb)] >> vb) << 4), "shared-memory slots"
        # a transpose marked warp-local waits at a warp barrier only: every
        # warp must read, in the new layout, exactly the local indices (hence
        # shared-memory slots) it wrote in the previous one
        for r in range(1, nr):
            stats.transposes += 1
            if int(rounds[r]["warp_local"]):
                stats.warp_local_transposes += 1
                a_w = np.sort(layouts[r - 1].reshape(-1, 32 * (1 << log_r)), axis=1)
                b_w = np.sort(layouts[r].reshape(-1, 32 * (1 << log_r)), axis=1)
                assert np.array_equal(a_w, b_w), "warp-local transpose moves keys between warps"
        for idx in (0, nr - 1):
            thr = rounds[idx]["thr_loc"]
            need = min(3, c - vb)
            if not all(int(thr[t]) == 1 << (vb + t) and int(P["gvec"][vb + t]) == 1 << (vb + t)
                       for t in range(need)):
                stats.uncoalesced_rounds += 1   # allowed only with io_direct
        G = _global_of_local(P["gvec"], m, np.arange(1 << m, dtype=np.int64))
        c = int(P["row_log"])
        assert c >= vb + 1 and all(int(P["gvec"][j]) == 1 << j for j in range(c))
        assert c == m or int(P["gvec"][c]) != 1 << c
        # the precomputed I/O vectors must agree with G on their rounds
        for io, rd in ((P["io"][0], rounds[0]), (P["io"][1], rounds[nr - 1])):
            for t in range(log_t):
                assert int(io["thr_glob"][t]) == int(G[int(rd["thr_loc"][t])])
            for j in range(log_r - vb):
                assert int(io["reg_glob"][j]) == int(G[int(rd["reg_loc"][j])])
        pos = g0[:, None] ^ G[None, :]                        # [cta, local]
        assert np.array_equal(np.sort(pos, axis=None), np.sort(np.unique(pos))), "tiles overlap"
        tile = a[pos]                                         # [cta, local] by local index
        regs = tile[:, layouts[0]]                            # [cta, thread, reg]
        _apply_steps(regs, rounds[0]["steps"][:rounds[0]["nsteps"]], desc)
        for r in range(1, nr):
            smem = np.empty_like(tile)
            smem[:, layouts[r - 1]] = regs
            regs = smem[:, layouts[r]]
            _apply_steps(regs, rounds[r]["steps"][:rounds[r]["nsteps"]], desc)
        out = np.empty_like(tile)
        out[:, layouts[nr - 1]] = regs
        a[pos] = out
    # virtual pads must still hold pad values (the kernel never stores them)
    assert np.all(a[:front] == front_pad), "front pad disturbed"
    assert np.all(a[front + n:N] == tail_pad), "tail pad disturbed"
    return a[front:front + n].copy(), plan, stats
