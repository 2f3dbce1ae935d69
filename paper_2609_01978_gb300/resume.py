"""Checkpoint / resume of one aperture in row groups (Fig. 18, Stage 2: chunk
groups and a resume manifest; verified groups are skipped on restart).

The focal-plane field is a sum over aperture rows (Sec. 2.6), so a group of
rows is checkpointed as its partial focal-plane field -- M x M complex, 16 M^2
bytes -- rather than as its row intermediate: the column pass runs per group,
and restarting needs only the finished groups' partial fields.  The run
directory holds one ``group_<k>.npy`` per finished group and ``manifest.json``:
the problem's fingerprint, the group layout and, per finished group, its rows
and the SHA-256 of its file.  A group whose file is missing or does not match
its checksum is computed again; a manifest written for another problem or
another layout is refused.

The partial field of a group comes from a callable ``propagate(j0, j1)`` that
returns the M x M complex field of rows [j0, j1) as a host array; ``plan_source``
builds it from a ``Plan`` (device propagation, one copy to host per group).
"""
from __future__ import annotations

import hashlib
import json
import os
import shutil
from typing import Callable, Optional

import numpy as np

MANIFEST = "manifest.json"


def fingerprint(params: dict) -> str:
    """Stable digest of the problem's parameters (any JSON-serialisable dict)."""
    blob = json.dumps(params, sort_keys=True, separators=(",", ":")).encode()
    return hashlib.sha256(blob).hexdigest()


def groups(jlo: int, jhi: int, group_rows: int) -> list:
    """Contiguous groups of `group_rows` rows covering [jlo, jhi)."""
    if group_rows < 1:
        raise ValueError("group_rows must be >= 1")
    return [(j, min(j + group_rows, jhi)) for j in range(jlo, jhi, group_rows)]


def _sha256(path: str) -> str:
    h = hashlib.sha256()
    with open(path, "rb") as fh:
        for block in iter(lambda: fh.read(1 << 20), b""):
            h.update(block)
    return h.hexdigest()


def _write_json(path: str, obj) -> None:
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(obj, fh, indent=1, sort_keys=True)
        fh.flush()
        os.fsync(fh.fileno())
    os.replace(tmp, path)


class GroupRun:
    """Row-group checkpointing of one propagation.

    ``run()`` computes every group that is not yet verified on disk, writing its
    partial field and updating the manifest after each group, and returns the
    summed field.  Interrupting it (an exception, a killed process) loses at
    most the group in flight."""

    def __init__(self, out_dir: str, params: dict, M: int, jlo: int, jhi: int, group_rows: int):
        self.out_dir = out_dir
        self.M = M
        self.layout = {"jlo": jlo, "jhi": jhi, "group_rows": group_rows, "M": M}
        self.fp = fingerprint(params)
        self.params = params
        self.groups = groups(jlo, jhi, group_rows)
        os.makedirs(out_dir, exist_ok=True)
        self.manifest_path = os.path.join(out_dir, MANIFEST)
        self.manifest = self._load()

    # -- manifest
    def _load(self) -> dict:
        if not os.path.exists(self.manifest_path):
            return {"fingerprint": self.fp, "params": self.params, "layout": self.layout, "done": {}}
        with open(self.manifest_path) as fh:
            m = json.load(fh)
        if m.get("fingerprint") != self.fp:
            raise ValueError(f"{self.manifest_path} belongs to another problem")
        if m.get("layout") != self.layout:
            raise ValueError(f"{self.manifest_path} has another group layout: {m.get('layout')}")
        return m

    def _file(self, k: int) -> str:
        return os.path.join(self.out_dir, f"group_{k:06d}.npy")

    def verified(self, k: int) -> bool:
        """Group k is recorded, its file exists and matches its checksum."""
        rec = self.manifest["done"].get(str(k))
        path = self._file(k)
        if rec is None or not os.path.exists(path):
            return False
        return rec.get("rows") == list(self.groups[k]) and rec.get("sha256") == _sha256(path)

    def pending(self) -> list:
        return [k for k in range(len(self.groups)) if not self.verified(k)]

    def preflight(self) -> None:
        """Refuse to start when the disk cannot hold the remaining groups."""
        need = len(self.pending()) * (16 * self.M * self.M + 4096)
        free = shutil.disk_usage(self.out_dir).free
        if free < need:
            raise OSError(f"{self.out_dir}: {free} bytes free, {need} needed for the remaining groups")

    # -- run
    def run(self, propagate: Callable[[int, int], np.ndarray],
            on_group: Optional[Callable[[int], None]] = None) -> np.ndarray:
        self.preflight()
        for k in self.pending():
            j0, j1 = self.groups[k]
            part = np.ascontiguousarray(propagate(j0, j1), dtype=np.complex128)
            if part.shape != (self.M, self.M):
                raise ValueError(f"partial field of group {k} has shape {part.shape}")
            path = self._file(k)
            tmp = path + ".tmp"
            with open(tmp, "wb") as fh:
                np.save(fh, part)
                fh.flush()
                os.fsync(fh.fileno())
            os.replace(tmp, path)
            self.manifest["done"][str(k)] = {"rows": [j0, j1], "sha256": _sha256(path)}
            _write_json(self.manifest_path, self.manifest)
            if on_group is not None:
                on_group(k)
        return self.total()

    def total(self) -> np.ndarray:
        """Sum of the verified groups' partial fields (all groups must be done)."""
        missing = self.pending()
        if missing:
            raise RuntimeError(f"groups not finished: {missing[:8]}{'...' if len(missing) > 8 else ''}")
        U = np.zeros((self.M, self.M), dtype=np.complex128)
        for k in range(len(self.groups)):
            U += np.load(self._file(k))
        return U


def plan_source(plan, torch, device=None) -> Callable[[int, int], np.ndarray]:
    """propagate(j0, j1) for a ``Plan``: the rows' partial field on the device,
    copied to the host."""
    dev = device or torch.device("cuda")
    U = torch.empty((plan.M, plan.M), dtype=torch.complex128, device=dev)

    def propagate(j0: int, j1: int) -> np.ndarray:
        plan.propagate_roi(j0, j1, U)
        return U.cpu().numpy()

    return propagate
