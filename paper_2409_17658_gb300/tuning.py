"""The tuning table kept in a JSON file.

The library holds the autotuners' results in a process-wide table (include/rd.h, rd_tune_*): the
split-K factor of the dense product per size class, the row-split passes' slab widths and slabs per
CTA per (m, j), and the sparse step's rows per block per size class.  This module saves that table
to a JSON file and loads it back, so a tuned shape outlives the process:

    {"format": "rd-tune-1", "device": "<GPU name>", "entries": [
        {"mode": "gemm_splitk", "key": 10, "aux": 10, "p": [8, 0, 0, 0], "ms": 0.0506}, ...]}

Entries of another device are skipped on load (a launch shape tuned on one GPU says little about
another); loading never changes results, only launch shapes.
"""
from __future__ import annotations

import json

from . import tune_set, tune_table

FORMAT = "rd-tune-1"


def _device_name() -> str:
    import torch

    return torch.cuda.get_device_name(torch.cuda.current_device()) if torch.cuda.is_available() else "cpu"


def save(path: str, device: str | None = None) -> dict:
    """Write the library's current table to path; returns the document written."""
    doc = {"format": FORMAT, "device": device if device is not None else _device_name(), "entries": tune_table()}
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)
    return doc


def load(path: str, device: str | None = None, merge: bool = True) -> int:
    """Install the entries of a saved table (those of this device); merge keeps the current entries
    whose keys the file does not have.  Returns the number of entries installed from the file."""
    with open(path) as f:
        doc = json.load(f)
    if doc.get("format") != FORMAT:
        raise ValueError(f"{path}: not a tuning table ({doc.get('format')!r})")
    dev = device if device is not None else _device_name()
    if doc.get("device") != dev:
        return 0
    new = list(doc["entries"])
    keys = {(e["mode"], e["key"], e["aux"]) for e in new}
    cur = [e for e in tune_table() if (e["mode"], e["key"], e["aux"]) not in keys] if merge else []
    tune_set(cur + new)
    return len(new)
