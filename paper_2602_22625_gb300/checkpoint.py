"""Checkpoint and resume of an optimisation: the primitive parameters, the Adam
moments and the step counter (plus any other named arrays) in one file.

Format (little-endian throughout):
    8 bytes   magic b"DBMPCKPT"
    4 bytes   format version (uint32, 1)
    4 bytes   header length L (uint32)
    L bytes   UTF-8 JSON header: {"step": int, "meta": {...}, "arrays": [{"name", "dtype",
              "shape", "offset", "nbytes"}, ...]}, offsets counted from the end of the header
    ...       the arrays' raw little-endian bytes, C order, each at its offset

Device tensors are copied to the host on save; `load` returns numpy arrays, which the
caller copies back to the device.  Arrays come back bit for bit, so a resumed run
continues from exactly the saved state.
"""
import json
import os
import struct

import numpy as np

MAGIC = b"DBMPCKPT"
VERSION = 1
_DTYPES = {"float32": "<f4", "float64": "<f8", "int32": "<i4", "int64": "<i8", "uint8": "|u1"}


def _to_numpy(a):
    if hasattr(a, "detach"):        # torch tensor, on any device
        a = a.detach().cpu().numpy()
    a = np.ascontiguousarray(a)
    if a.dtype.name not in _DTYPES:
        raise TypeError(f"unsupported dtype {a.dtype}")
    return a.astype(_DTYPES[a.dtype.name], copy=False)


def save(path, arrays, step, meta=None):
    """Writes `arrays` (name -> numpy array or torch tensor), the step counter and a
    JSON-serialisable `meta` dict to `path` (atomically: a temporary file is renamed)."""
    entries, blobs, off = [], [], 0
    for name, a in arrays.items():
        a = _to_numpy(a)
        b = a.tobytes(order="C")
        entries.append({"name": name, "dtype": np.dtype(a.dtype).name, "shape": list(a.shape), "offset": off,
                        "nbytes": len(b)})
        blobs.append(b)
        off += len(b)
    header = json.dumps({"step": int(step), "meta": meta or {}, "arrays": entries}).encode("utf-8")
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<II", VERSION, len(header)))
        f.write(header)
        for b in blobs:
            f.write(b)
    os.replace(tmp, path)


def load(path):
    """Returns (arrays: name -> numpy array, step, meta) from a file `save` wrote."""
    with open(path, "rb") as f:
        data = f.read()
    if data[:8] != MAGIC:
        raise ValueError(f"{path}: not a checkpoint (bad magic)")
    version, hlen = struct.unpack_from("<II", data, 8)
    if version != VERSION:
        raise ValueError(f"{path}: checkpoint version {version}, expected {VERSION}")
    header = json.loads(data[16:16 + hlen].decode("utf-8"))
    base = 16 + hlen
    arrays = {}
    for e in header["arrays"]:
        start, n = base + e["offset"], e["nbytes"]
        if start + n > len(data):
            raise ValueError(f"{path}: truncated array {e['name']}")
        dt = np.dtype(_DTYPES[e["dtype"]])
        arrays[e["name"]] = np.frombuffer(data, dtype=dt, count=n // dt.itemsize, offset=start).reshape(
            e["shape"]).copy()
    return arrays, header["step"], header["meta"]
