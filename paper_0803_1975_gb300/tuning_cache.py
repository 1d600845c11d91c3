"""Persistent cache of the autotuners' choices, a JSON file.

The dot-form autotuner (gfp_dot_autotune) and the batched autotuner
(gfp_batched_autotune) time candidates on the GPU; their choices depend only
on the shapes, the library build and the GPU.  This cache keeps them across
processes: an entry is reused when the file was written by the same library
build (a hash of libgfp.so) on a GPU of the same name, and the whole file is
discarded -- rebuilt on the next tuning -- when either differs.

    cache = TuningCache("gfp_tuning.json")
    best = cache.dot(p, m, k, n)                  # (word, d, Q, kb), timed once
    cache.batched(probs, count)                   # installs the batched table

Host-side bookkeeping only: the choices are made and used by the library.
"""
from __future__ import annotations

import hashlib
import json
import os
import tempfile

from . import gfp

VERSION = 1


def library_stamp(path: str | None = None) -> str:
    """Short hash of the library file: a rebuilt library invalidates the cache."""
    h = hashlib.sha256()
    with open(path or gfp.lib_path(), "rb") as f:
        for chunk in iter(lambda: f.read(1 << 20), b""):
            h.update(chunk)
    return h.hexdigest()[:16]


def batch_signature(problems) -> str:
    """The batched autotuner's choice depends on how many problems fall in
    each size bucket and whether p < 16 (the tcgen05 tiles): this multiset,
    as a string."""
    counts = {}
    for p, m, k, n in problems:
        s = max(m, k, n)
        b = 0 if s <= 32 else 1 if s <= 64 else 2 if s <= 128 else 3 if s <= 256 else 4 if s <= 512 else \
            5 if s <= 2048 else 6
        key = "%d%s" % (b, "t" if p < 16 else "h")
        counts[key] = counts.get(key, 0) + 1
    return ",".join("%s:%d" % kv for kv in sorted(counts.items()))


class TuningCache:
    def __init__(self, path: str, stamp: str | None = None, device: str | None = None):
        self.path = path
        self.stamp = stamp if stamp is not None else library_stamp()
        if device is None:
            import torch
            device = torch.cuda.get_device_name()
        self.device = device
        self.data = {"version": VERSION, "library": self.stamp, "device": self.device, "dot": {}, "batched": {}}
        self.reused = False
        try:
            with open(path) as f:
                old = json.load(f)
            if (old.get("version") == VERSION and old.get("library") == self.stamp
                    and old.get("device") == self.device):
                self.data["dot"] = dict(old.get("dot", {}))
                self.data["batched"] = dict(old.get("batched", {}))
                self.reused = True
        except (OSError, ValueError):
            pass

    def save(self):
        d = os.path.dirname(os.path.abspath(self.path))
        fd, tmp = tempfile.mkstemp(dir=d, prefix=".gfp_tuning_")
        with os.fdopen(fd, "w") as f:
            json.dump(self.data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def dot(self, p: int, m: int, k: int, n: int):
        """(word, d, Q, kb) of the dot form for this shape: from the cache, or
        timed by gfp_dot_autotune and stored."""
        key = "%d:%d:%d:%d" % (p, m, k, n)
        c = self.data["dot"].get(key)
        if c is None:
            best, _ = gfp.gfp_dot_autotune(p, m, k, n)
            c = {"word": best["word"], "d": best["d"], "Q": best["Q"], "kb": best["kb"], "ms": best["ms"]}
            self.data["dot"][key] = c
            self.save()
        return c["word"], c["d"], c["Q"], c["kb"]

    def batched(self, probs, count: int, workspace=None):
        """Install the batched table for this batch: from the cache
        (gfp_batched_set_table), or tuned by gfp_batched_autotune and stored.
        Returns the table."""
        sig = batch_signature((probs[i].p, probs[i].m, probs[i].k, probs[i].n) for i in range(count))
        table = self.data["batched"].get(sig)
        if table is None:
            table = gfp.gfp_batched_autotune(probs, count, workspace=workspace)
            self.data["batched"][sig] = list(table)
            self.save()
        else:
            gfp.gfp_batched_set_table(table)
        return list(table)
