"""Autotuner of the per-start kernel layout of the batched form.

Each start of a batch runs either on one lane (H of the start in the
block's shared memory, 32 starts to a warp), or on one warp (four starts to
a 128-thread block), or on one 128-thread block, or on lanes first with the
long runs handed over to blocks (the automatic choice for d <= 16).  Which is fastest depends on the objective, the
dimension, the precision and the gradient mode, and the arithmetic does not:
every layout produces the same bits (the kernels perform the same operations
in the same order), so the tuner only changes the time.

The tuner keys problems by (objective, dimension bucket, precision, gradient
mode), times every layout the kernels accept on a probe batch built from the
problems of that key (at most `probe_problems` of them, truncated to
`probe_starts` starts each, repeated with other seeds until the probe holds
`probe_total` starts, so that the layouts that keep many starts on an SM at
once are compared at throughput rather than at the latency of a few
starts), and keeps the fastest.  Choices persist in a
JSON file keyed also by the device name, so a key is measured once per GPU
model.  L-BFGS problems have one layout (a 256-thread block per start) and
are not tuned.
"""
from __future__ import annotations

import json
import os
import threading

# upper ends of the dimension buckets
BUCKETS = (2, 4, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 512, 1024, 4096)

# threads_per_start values the kernels provide: 0 automatic (lanes with
# hand-over for d <= 16, else a block), 1 lanes throughout, 32 a warp (four
# starts to a block), 128 a block
CANDIDATES = (0, 1, 32, 128)


def bucket(d: int) -> int:
    for b in BUCKETS:
        if d <= b:
            return b
    return BUCKETS[-1]


def default_cache_path() -> str:
    base = os.environ.get("ZEUS_AUTOTUNE_CACHE")
    if base:
        return base
    home = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(home, "zeus_gb300", "autotune.json")


class Autotuner:
    """Chooses threads_per_start per problem of a batch by measurement.

    measure(problems) -> milliseconds, if given, replaces the GPU timing
    (used by the host tests); by default a probe batch is solved on the
    current CUDA device and timed with CUDA events."""

    def __init__(self, cache_path: str | None = None, probe_problems: int = 16,
                 probe_starts: int = 256, reps: int = 1, measure=None, device_name: str | None = None,
                 probe_total: int = 8192):
        self.cache_path = cache_path or default_cache_path()
        self.probe_problems = probe_problems
        self.probe_starts = probe_starts
        self.probe_total = probe_total
        self.reps = reps
        self._measure = measure or self._measure_gpu
        self._device = device_name
        self._lock = threading.Lock()
        self.table = self._load()

    # -------------------------------------------------------------- keys
    @staticmethod
    def key(p) -> str:
        return f"obj{int(p.objective)}/d{bucket(int(p.dim))}/prec{int(p.precision)}/grad{int(p.grad_mode)}"

    def device_name(self) -> str:
        if self._device is None:
            import torch
            self._device = torch.cuda.get_device_name() if torch.cuda.is_available() else "none"
        return self._device

    # ------------------------------------------------------------- cache
    def _load(self) -> dict:
        try:
            with open(self.cache_path) as fh:
                t = json.load(fh)
            return t if isinstance(t, dict) else {}
        except (OSError, ValueError):
            return {}

    def save(self) -> None:
        d = os.path.dirname(self.cache_path)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = f"{self.cache_path}.tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(self.table, fh, indent=1, sort_keys=True)
        os.replace(tmp, self.cache_path)

    def choice(self, p) -> int | None:
        e = self.table.get(self.device_name(), {}).get(self.key(p))
        return None if e is None else int(e["threads_per_start"])

    # ------------------------------------------------------------ tuning
    @staticmethod
    def _valid(p, tps: int) -> bool:
        from . import _capi, zeus_plan_info, zeus_validate
        q = _capi.zeus_problem.from_buffer_copy(bytes(p))
        q.threads_per_start = tps
        if zeus_validate(q) != 0:
            return False
        try:
            plan = zeus_plan_info(q)
        except _capi.ZeusError:
            return False
        return not plan["stream"]  # the batch holds H on chip

    def _probe(self, members, tps: int):
        from . import _capi
        out, total, r = [], 0, 0
        base = members[: self.probe_problems]
        while True:
            for p in base:
                q = _capi.zeus_problem.from_buffer_copy(bytes(p))
                q.threads_per_start = tps
                q.n_starts = min(int(q.n_starts), self.probe_starts)
                q.seed = (int(q.seed) + 1000003 * r) & (2**64 - 1)
                out.append(q)
                total += int(q.n_starts)
            r += 1
            if total >= self.probe_total or r >= 64:
                return out

    def _measure_gpu(self, probe) -> float:
        import torch

        from . import Batch
        b = Batch(probe)
        b.solve()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = float("inf")
        for _ in range(self.reps):
            e0.record()
            b.solve()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    def tune(self, problems) -> dict:
        """Measure every key of `problems` not in the cache; returns
        {key: threads_per_start} for all their keys."""
        from . import _prob
        problems = [_prob(p) for p in problems]
        groups: dict[str, list] = {}
        for p in problems:
            groups.setdefault(self.key(p), []).append(p)
        dev = self.device_name()
        with self._lock:
            entries = self.table.setdefault(dev, {})
            changed = False
            for k, members in groups.items():
                if k in entries:
                    continue
                cands = [c for c in CANDIDATES if all(self._valid(p, c) for p in members)]
                if not cands:
                    continue
                times = {c: self._measure(self._probe(members, c)) for c in cands}
                best = min(cands, key=lambda c: (times[c], c))
                entries[k] = {"threads_per_start": best,
                              "ms": {str(c): round(t, 4) for c, t in times.items()},
                              "probe": f"{min(len(members), self.probe_problems)} problems x "
                                       f"<= {self.probe_starts} starts"}
                changed = True
            if changed:
                self.save()
        return {k: int(entries[k]["threads_per_start"]) for k in groups if k in entries}

    def apply(self, problems, tune: bool = True):
        """Copies of `problems` with threads_per_start set from the table
        (measuring missing keys first if `tune`); problems that set
        threads_per_start themselves keep it."""
        from . import _capi, _prob
        problems = [_prob(p) for p in problems]
        if tune:
            self.tune([p for p in problems if p.threads_per_start == 0 and p.lbfgs_m == 0])
        out = []
        for p in problems:
            q = _capi.zeus_problem.from_buffer_copy(bytes(p))
            if q.threads_per_start == 0 and q.lbfgs_m == 0:  # L-BFGS has one layout
                c = self.choice(q)
                if c is not None:
                    q.threads_per_start = c
            out.append(q)
        return out
