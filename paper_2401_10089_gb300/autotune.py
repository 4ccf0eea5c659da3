"""Autotuner for the batching form: per size bucket, the kernel configuration
of the one-block-per-matrix path that runs a batch fastest on this GPU.

For every size bucket present in the batch (n <= 8, 16, 32, 64, 128, 256) the
tuner takes the batch's matrices of that bucket (up to ``sample``), times
``logm_execute`` on them with each configuration the bucket can use (CUDA
events, median of ``reps`` after a warm-up), keeps the fastest, and finally
installs the table (``set_tuning``) and optionally writes it to JSON. The
binding loads ``tuning_gb300.json`` next to this file when the library is
first loaded.

    python -m paper_2401_10089_gb300.autotune --out paper_2401_10089_gb300/tuning_gb300.json
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import api

BUCKET_MAX_N = (8, 16, 32, 64, 128, 256)
# configurations: 0 = 256 threads, n <= 256; 1 = 128 threads, n <= 64; 2 = 64 threads,
# n <= 32; 3 = 256 threads, three blocks per SM; 4 = configuration 2 with the working
# matrices in shared memory
CANDIDATES = {0: (0, 1, 2, 4), 1: (0, 1, 2, 4), 2: (0, 1, 2, 4), 3: (0, 1, 3), 4: (0, 3), 5: (0, 3)}


def _bucket(n: int) -> int:
    for b, m in enumerate(BUCKET_MAX_N):
        if n <= m:
            return b
    return len(BUCKET_MAX_N)


def _sub_batch(A, idx):
    """The matrices idx of a Ragged or (count, n, n) batch, as a new batch."""
    if not isinstance(A, api.Ragged):
        return A[torch.as_tensor(idx, device=A.device)].contiguous()
    ns = A.n.cpu().numpy()[idx]
    offs = A.offset.cpu().numpy()[idx]
    vals = torch.cat([A.values[int(o):int(o) + int(n) * int(n)] for o, n in zip(offs, ns)])
    new_off = np.zeros(len(idx), dtype=np.int64)
    new_off[1:] = np.cumsum(ns.astype(np.int64) ** 2)[:-1]
    dev = A.values.device
    return api.Ragged(vals, torch.as_tensor(ns, dtype=torch.int32, device=dev),
                      torch.as_tensor(new_off, device=dev), int(ns.max()))


def _time(fn, reps):
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def pick(times_ms: dict, margin: float = 0.02) -> int:
    """Configuration 0 unless another is faster by more than ``margin`` (a
    configuration that only ties is noise on one batch and can lose on
    another: three 256-thread blocks per SM balance unequal matrices worse)."""
    best = min(times_ms, key=times_ms.get)
    if 0 in times_ms and times_ms[best] > (1.0 - margin) * times_ms[0]:
        return 0
    return best


def autotune(A, precision: str = "fp64", sample: int = 4096, reps: int = 3, path: str | None = None,
             margin: float = 0.02):
    """Tune the per-bucket configuration on batch A; returns (table, times_ms)."""
    if isinstance(A, api.Ragged):
        ns = A.n.cpu().numpy()
    else:
        ns = np.full(A.shape[0], A.shape[-1], dtype=np.int32)
    table = api.get_tuning()
    times = {}
    for bk in range(len(BUCKET_MAX_N)):
        idx = np.nonzero([_bucket(int(n)) == bk for n in ns])[0][:sample]
        if len(idx) == 0:
            continue
        sub = _sub_batch(A, idx)
        res = {}
        for v in CANDIDATES[bk]:
            trial = list(table)
            trial[bk] = v
            api.set_tuning(trial)
            res[v] = _time(lambda: api.logm_execute(sub, precision=precision), reps)
        table[bk] = pick(res, margin)
        times[BUCKET_MAX_N[bk]] = {str(v): t for v, t in res.items()}
    api.set_tuning(table)
    if path:
        with open(path, "w") as f:
            json.dump({"variant": table, "buckets_max_n": list(BUCKET_MAX_N), "precision": precision, "margin": margin,
                       "device": torch.cuda.get_device_name(), "times_ms": times,
                       "variants": {"0": "256 threads, 64x64 DMMA tiles, n <= 256",
                                    "1": "128 threads, 32x32 tiles, n <= 64",
                                    "2": "64 threads, 32x32 tiles, n <= 32",
                                    "3": "256 threads, 64x64 tiles, n <= 256, 3 blocks per SM",
                                    "4": "64 threads, 32x32 tiles, n <= 32, working matrices in shared memory"}},
                      f, indent=1)
    return table, times


def main():
    from . import workloads
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=7000, help="ragged SPD matrices, n uniform over {4, 8, ..., 256} (powers of two)")
    ap.add_argument("--precision", default="fp64")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    vals, ns, offs = workloads.ragged_spd(args.count)
    dev = torch.device("cuda")
    R = api.Ragged(torch.from_numpy(vals).to(dev), torch.from_numpy(ns).to(dev), torch.from_numpy(offs).to(dev), 256)
    api.set_tuning(None)
    table, times = autotune(R, precision=args.precision, path=args.out)
    print(json.dumps({"variant": table, "times_ms": times}))


if __name__ == "__main__":
    main()
