"""Continuous-batching sort server driving the C ABI.

Requests (uint32 keys, some with uint32 values) arrive over time.  The loop:

  * admits requests in arrival order while their device buffers fit a memory
    budget (a first-fit arena carved out of one resident device allocation)
    and their results fit the pinned host output area;
  * packs the admitted small requests (at most one packed tile: 16K keys or
    8K pairs) into one segmented launch per kind
    (bitonic_sort_segmented_u32 / bitonic_sort_segmented_pairs_u32_bounded),
    and gives every larger request its own bitonic_sort_u32 /
    bitonic_sort_pairs_u32 launch;
  * spreads launches round-robin over several CUDA streams, so requests that
    arrive while others are on the GPU are admitted and run concurrently;
  * copies inputs host -> device and results device -> host on the same
    stream, records an event, and polls events to detect completion, freeing
    the request's buffers and timestamping it on the host monotonic clock.

Latency = completion - arrival, including queueing.  The sorts themselves are
the library's CUDA kernels.  By default the loop runs inside the library
(bitonic_serve_run: one C++ host thread, plain CUDA runtime calls per copy
and launch); this module sets up the buffers and streams, warms the plans up
and computes the statistics.  The same loop written in Python
(engine="python") is kept for comparison: at high request rates its
per-call overhead, not the GPU, sets the latency.
"""
from __future__ import annotations

import ctypes
import time
from dataclasses import dataclass, field

import numpy as np

from . import load, OK, status_string, thread_graphs, ServeConfig, ServeStats, serve_request_dtype

ALIGN = 16


class Arena:
    """First-fit allocator over [0, size) in ALIGN-byte units (host bookkeeping)."""

    def __init__(self, size: int):
        self.size = size
        self.free = [(0, size)]  # sorted (offset, length)
        self.used = 0
        self.peak = 0

    def alloc(self, nbytes: int):
        nbytes = (nbytes + ALIGN - 1) // ALIGN * ALIGN
        for i, (off, ln) in enumerate(self.free):
            if ln >= nbytes:
                if ln == nbytes:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + nbytes, ln - nbytes)
                self.used += nbytes
                self.peak = max(self.peak, self.used)
                return off, nbytes
        return None

    def release(self, block):
        off, nbytes = block
        self.used -= nbytes
        # insert and coalesce with neighbours
        lo, hi = 0, len(self.free)
        while lo < hi:
            mid = (lo + hi) // 2
            if self.free[mid][0] < off:
                lo = mid + 1
            else:
                hi = mid
        self.free.insert(lo, (off, nbytes))
        if lo + 1 < len(self.free) and self.free[lo][0] + self.free[lo][1] == self.free[lo + 1][0]:
            self.free[lo] = (off, self.free[lo][1] + self.free[lo + 1][1])
            self.free.pop(lo + 1)
        if lo > 0 and self.free[lo - 1][0] + self.free[lo - 1][1] == self.free[lo][0]:
            self.free[lo - 1] = (self.free[lo - 1][0], self.free[lo - 1][1] + self.free[lo][1])
            self.free.pop(lo)


@dataclass
class Request:
    idx: int
    arrival: float          # seconds since the start of the run
    n: int                  # keys
    has_vals: bool
    src: int                # first key in the host input pool
    admit: float = -1.0
    done: float = -1.0
    out: int = -1           # first key of its result in the host output area
    blocks: list = field(default_factory=list)


@dataclass
class Flight:
    event: object
    requests: list
    dev_blocks: list
    host_blocks: list


class SortServer:
    """Sort server over one device-memory budget.

    pool_keys / pool_vals: uint32 numpy arrays the requests' inputs are read
    from (the three request kinds -- small keys, small pairs, large -- each
    take consecutive slices of their own third of the pool, wrapping around).
    """

    def __init__(self, pool_keys: np.ndarray, pool_vals: np.ndarray, budget_bytes: int = 16 << 30,
                 streams: int = 4, out_keys: int | None = None, small_keys: int = 1 << 14,
                 small_pairs: int = 1 << 13, max_batch: int = 1024):
        import torch

        self.torch = torch
        self.lib = load()
        self.budget = int(budget_bytes)
        self.dev = torch.empty(self.budget, dtype=torch.uint8, device="cuda")  # resident arena
        self.dev_base = self.dev.data_ptr()
        self.arena = Arena(self.budget)
        n_pool = pool_keys.size
        self.in_keys = torch.from_numpy(np.ascontiguousarray(pool_keys).view(np.int32)).pin_memory()
        self.in_vals = torch.from_numpy(np.ascontiguousarray(pool_vals).view(np.int32)).pin_memory()
        n_out = out_keys or n_pool
        self.out_keys = torch.empty(n_out, dtype=torch.int32).pin_memory()
        self.out_vals = torch.empty(n_out, dtype=torch.int32).pin_memory()
        self.host_arena = Arena(n_out * 4)
        self.offs_stage = torch.empty(1 << 20, dtype=torch.int32).pin_memory()
        self.offs_cursor = 0
        self.streams = [torch.cuda.Stream() for _ in range(streams)]
        self.small_keys, self.small_pairs, self.max_batch = small_keys, small_pairs, max_batch
        third = n_pool // 3
        self.rings = {"sk": [0, third], "sp": [third, third], "lg": [2 * third, n_pool - 2 * third]}
        self.ring_pos = {k: 0 for k in self.rings}

    # -- request bookkeeping -------------------------------------------------
    def _kind(self, n, has_vals):
        if has_vals:
            return "sp" if n <= self.small_pairs else "lg"
        return "sk" if n <= self.small_keys else "lg"

    def _src(self, kind, n):
        base, size = self.rings[kind]
        if n > size:
            raise ValueError(f"request of {n} keys exceeds the input pool")
        pos = self.ring_pos[kind]
        if pos + n > size:
            pos = 0
        self.ring_pos[kind] = pos + n
        return base + pos

    def _stream(self):
        s = self.streams[self._rr % len(self.streams)]
        self._rr += 1
        return s

    def _offsets_to_device(self, offs: np.ndarray, dev_off: int, stream):
        n = offs.size
        if self.offs_cursor + n > self.offs_stage.numel():
            self.offs_cursor = 0
        stage = self.offs_stage[self.offs_cursor:self.offs_cursor + n]
        self.offs_cursor += n
        stage.numpy()[:] = offs
        dst = self.dev[dev_off:dev_off + 4 * n].view(self.torch.int32)
        with self.torch.cuda.stream(stream):
            dst.copy_(stage, non_blocking=True)
        return dst

    # -- launches --------------------------------------------------------------
    def _copy_in(self, reqs, key_off, val_off, stream):
        """H2D copies of consecutive requests' inputs (one copy per contiguous run)."""
        torch = self.torch
        with torch.cuda.stream(stream):
            dev_pos = 0
            i = 0
            while i < len(reqs):
                j = i + 1
                while j < len(reqs) and reqs[j].src == reqs[j - 1].src + reqs[j - 1].n:
                    j += 1
                src, n = reqs[i].src, sum(r.n for r in reqs[i:j])
                dk = self.dev[key_off + 4 * dev_pos:key_off + 4 * (dev_pos + n)].view(torch.int32)
                dk.copy_(self.in_keys[src:src + n], non_blocking=True)
                if val_off is not None:
                    dv = self.dev[val_off + 4 * dev_pos:val_off + 4 * (dev_pos + n)].view(torch.int32)
                    dv.copy_(self.in_vals[src:src + n], non_blocking=True)
                dev_pos += n
                i = j

    def _launch(self, reqs, kind):
        """Allocates, copies in, sorts, copies out; returns a Flight or None."""
        torch = self.torch
        total = sum(r.n for r in reqs)
        pairs = kind == "sp" or (kind == "lg" and reqs[0].has_vals)
        batch = kind in ("sk", "sp")
        dev_bytes = 4 * total * (2 if pairs else 1) + (4 * (len(reqs) + 1) if batch else 0) + 3 * 16
        dblk = self.arena.alloc(dev_bytes)
        if dblk is None:
            return None
        hblk = self.host_arena.alloc(4 * total)
        if hblk is None:
            self.arena.release(dblk)
            return None
        stream = self._stream()
        base = dblk[0]
        key_off = base
        val_off = base + (4 * total + 15) // 16 * 16 if pairs else None
        offs_off = (val_off if pairs else key_off) + (4 * total + 15) // 16 * 16
        self._copy_in(reqs, key_off, val_off, stream)
        kptr = self.dev_base + key_off
        vptr = self.dev_base + val_off if pairs else None
        sh = stream.cuda_stream
        if batch:
            offs = np.zeros(len(reqs) + 1, dtype=np.int32)
            np.cumsum([r.n for r in reqs], out=offs[1:])
            d_offs = self._offsets_to_device(offs, offs_off, stream)
            if pairs:
                st = self.lib.bitonic_sort_segmented_pairs_u32_bounded(kptr, vptr, d_offs.data_ptr(), len(reqs),
                                                                       self.small_pairs, sh)
            else:
                st = self.lib.bitonic_sort_segmented_u32(kptr, d_offs.data_ptr(), len(reqs), sh)
        elif pairs:
            st = self.lib.bitonic_sort_pairs_u32(kptr, vptr, total, 1, sh)
        else:
            st = self.lib.bitonic_sort_u32(kptr, total, 1, sh)
        if st != OK:
            raise RuntimeError(f"sort launch failed: {status_string(st)}")
        out = hblk[0] // 4
        with torch.cuda.stream(stream):
            self.out_keys[out:out + total].copy_(self.dev[key_off:key_off + 4 * total].view(torch.int32),
                                                 non_blocking=True)
            if pairs:
                self.out_vals[out:out + total].copy_(self.dev[val_off:val_off + 4 * total].view(torch.int32),
                                                     non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        pos = out
        for r in reqs:
            r.out = pos
            pos += r.n
        return Flight(ev, list(reqs), [dblk], [hblk])

    def warmup(self, max_keys: int):
        """Before serving: sizes every stream's workspace and builds every plan
        up to max_keys, so no request pays for a cudaMalloc (which
        synchronises) or for host-side planning."""
        torch = self.torch
        with thread_graphs(False):
            n_max = min(max_keys, self.in_keys.numel())
            k = self.dev[:4 * n_max].view(torch.int32)
            v = self.dev[4 * n_max:8 * n_max].view(torch.int32)
            k.copy_(self.in_keys[:n_max])
            v.copy_(self.in_vals[:n_max])
            nb = max(1, min(self.max_batch, n_max))  # the largest packed batch sizes the segmented workspace
            offs = torch.arange(0, nb + 1, dtype=torch.int32, device="cuda") * min(self.small_pairs, n_max // nb)
            for stream in self.streams:
                sh = stream.cuda_stream
                with torch.cuda.stream(stream):
                    # every power of two up to the largest request, and the
                    # largest itself (its plan and its workspace size)
                    ns = [1 << j for j in range(10, 32) if (1 << j) <= n_max] + [n_max]
                    for n in ns:
                        for st in (self.lib.bitonic_sort_u32(k.data_ptr(), n, 1, sh),
                                   self.lib.bitonic_sort_pairs_u32(k.data_ptr(), v.data_ptr(), n, 1, sh)):
                            if st != OK:
                                raise RuntimeError(status_string(st))
                    for st in (self.lib.bitonic_sort_segmented_u32(k.data_ptr(), offs.data_ptr(), nb, sh),
                               self.lib.bitonic_sort_segmented_pairs_u32_bounded(
                                   k.data_ptr(), v.data_ptr(), offs.data_ptr(), nb, self.small_pairs, sh)):
                        if st != OK:
                            raise RuntimeError(status_string(st))
            torch.cuda.synchronize()

    # -- the loop --------------------------------------------------------------
    def run(self, arrival_s, sizes, has_vals, keep_outputs: bool = False, engine: str = "native"):
        """Serves the request stream; returns a statistics dict (and, with
        keep_outputs, the sorted keys / values of every request).

        engine "native": the loop runs in the library (bitonic_serve_run, one
        C++ host thread); "python": the same loop written here, one ctypes and
        torch call per copy and launch."""
        reqs = []
        for i, (a, n, hv) in enumerate(zip(arrival_s, sizes, has_vals)):
            kind = self._kind(int(n), bool(hv))
            reqs.append(Request(i, float(a), int(n), bool(hv), self._src(kind, int(n))))
        if engine == "native":
            return self._run_native(reqs, keep_outputs)
        if engine != "python":
            raise ValueError(f"unknown engine {engine!r}")
        return self._run_python(reqs, keep_outputs)

    def _stats(self, reqs, batch_sizes_sum, n_batches, n_large, peak, engine):
        lat = np.array([r.done - r.arrival for r in reqs])
        keys_total = int(sum(r.n for r in reqs))
        span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
        return {
            "requests": len(reqs), "keys": keys_total,
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3),
            "sustained_gkeys_s": keys_total / span / 1e9,
            "offered_gkeys_s": keys_total / max(reqs[-1].arrival, 1e-9) / 1e9,
            "batches": n_batches, "mean_batch": batch_sizes_sum / n_batches if n_batches else 0.0,
            "large_launches": n_large, "peak_device_bytes": peak, "budget_bytes": self.budget,
            "streams": len(self.streams), "engine": engine,
        }

    def _run_native(self, reqs, keep_outputs):
        torch = self.torch
        N = len(reqs)
        rq = np.zeros(N, dtype=serve_request_dtype())
        rq["arrival_s"] = [r.arrival for r in reqs]
        rq["src"] = [r.src for r in reqs]
        rq["n"] = [r.n for r in reqs]
        rq["has_vals"] = [int(r.has_vals) for r in reqs]
        if keep_outputs:
            # every result keeps its own place: one area for the whole stream
            total = int(sum((r.n + 3) // 4 * 4 for r in reqs))
            out_k = torch.empty(total, dtype=torch.int32).pin_memory()
            out_v = torch.empty(total, dtype=torch.int32).pin_memory()
        else:
            out_k, out_v = self.out_keys, self.out_vals
        handles = (ctypes.c_void_p * len(self.streams))(*[st.cuda_stream for st in self.streams])
        cfg = ServeConfig(dev_arena=self.dev_base, dev_bytes=self.budget,
                          in_keys=self.in_keys.data_ptr(), in_vals=self.in_vals.data_ptr(),
                          pool_len=self.in_keys.numel(), out_keys=out_k.data_ptr(), out_vals=out_v.data_ptr(),
                          out_cap=out_k.numel(), offs_stage=self.offs_stage.data_ptr(),
                          offs_cap=self.offs_stage.numel(), streams=handles, nstreams=len(self.streams),
                          small_keys=self.small_keys, small_pairs=self.small_pairs, max_batch=self.max_batch,
                          keep_outputs=int(bool(keep_outputs)))
        done = np.zeros(N, dtype=np.float64)
        pos = np.zeros(N, dtype=np.uint64)
        st = ServeStats()
        torch.cuda.synchronize()
        status = self.lib.bitonic_serve_run(ctypes.byref(cfg), rq.ctypes.data, N, done.ctypes.data,
                                            pos.ctypes.data, ctypes.byref(st))
        if status != OK:
            raise RuntimeError(f"bitonic_serve_run failed: {status_string(status)}")
        for r, d, p in zip(reqs, done, pos):
            r.done, r.out = float(d), int(p)
        stats = self._stats(reqs, st.batched_requests, st.batches, st.large_launches, st.peak_device_bytes,
                            "native")
        if not keep_outputs:
            return stats
        ok, ov = out_k.numpy().view(np.uint32), out_v.numpy().view(np.uint32)
        outputs = [(ok[r.out:r.out + r.n].copy(), ov[r.out:r.out + r.n].copy() if r.has_vals else None)
                   for r in reqs]
        return stats, outputs

    def _run_python(self, reqs, keep_outputs):
        torch = self.torch
        self._rr = 0
        N = len(reqs)
        outputs = [None] * N if keep_outputs else None
        pending, inflight = [], []
        nxt, done, n_batches, n_large, batch_sizes = 0, 0, 0, 0, []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # every launch has fresh buffers, so no cached graph would be replayed:
        # plain launches, for this thread's calls only
        with thread_graphs(False):
            while done < N:
                now = time.perf_counter() - t0
                while nxt < N and reqs[nxt].arrival <= now:
                    pending.append(reqs[nxt])
                    nxt += 1
                # admit in arrival order: small requests grouped per kind, large alone
                groups = {"sk": [], "sp": []}
                keep = []
                blocked = False
                for r in pending:
                    if blocked:
                        keep.append(r)
                        continue
                    kind = self._kind(r.n, r.has_vals)
                    if kind == "lg":
                        fl = self._launch([r], "lg")
                        if fl is None:
                            blocked = True
                            keep.append(r)
                            continue
                        r.admit = now
                        inflight.append(fl)
                        n_large += 1
                    else:
                        g = groups[kind]
                        g.append(r)
                        if len(g) == self.max_batch:
                            fl = self._launch(g, kind)
                            if fl is None:
                                blocked = True
                                keep.extend(g)
                            else:
                                for q in g:
                                    q.admit = now
                                inflight.append(fl)
                                n_batches += 1
                                batch_sizes.append(len(g))
                            groups[kind] = []
                for kind, g in groups.items():
                    if not g:
                        continue
                    fl = self._launch(g, kind) if not blocked else None
                    if fl is None:
                        keep.extend(g)
                        blocked = True
                    else:
                        for q in g:
                            q.admit = now
                        inflight.append(fl)
                        n_batches += 1
                        batch_sizes.append(len(g))
                keep.sort(key=lambda r: r.idx)
                pending = keep
                # completions
                still = []
                for fl in inflight:
                    if fl.event.query():
                        t = time.perf_counter() - t0
                        for r in fl.requests:
                            r.done = t
                            if keep_outputs:
                                k = self.out_keys[r.out:r.out + r.n].numpy().view(np.uint32).copy()
                                v = (self.out_vals[r.out:r.out + r.n].numpy().view(np.uint32).copy()
                                     if r.has_vals else None)
                                outputs[r.idx] = (k, v)
                        done += len(fl.requests)
                        for b in fl.dev_blocks:
                            self.arena.release(b)
                        for b in fl.host_blocks:
                            self.host_arena.release(b)
                    else:
                        still.append(fl)
                inflight = still
                if not pending and not inflight and nxt < N:
                    wait = reqs[nxt].arrival - (time.perf_counter() - t0)
                    if wait > 2e-4:
                        time.sleep(wait - 1e-4)
        stats = self._stats(reqs, float(sum(batch_sizes)), n_batches, n_large, self.arena.peak, "python")
        return (stats, outputs) if keep_outputs else stats
