"""Checkpoints of the staged workflow: ground state -> ACE -> Casida, and network training.

The paper's workflow runs in stages (a ground-state run, then the unoccupied states, then
the Casida solve), each starting from the last one's results.  A checkpoint file here is a
sequence of named arrays, each record

    magic  b"RSXC"          4 bytes
    version                 uint32 (1)
    name length, name       uint32, UTF-8 bytes
    dtype code              uint32 (0 float32, 1 float64, 2 int32, 3 int64, 4 bfloat16 bits as uint16)
    ndim, shape             uint32, ndim x int64
    payload bytes           uint64
    payload                 the array, C order, little-endian

all integers little-endian.  Arrays may be device tensors (copied to the host), host
tensors or numpy arrays; `load` returns numpy arrays, or tensors on `device`.  A record
whose magic, version or payload size does not check out raises ValueError (a truncated or
foreign file is never read as data).
"""
import struct

import numpy as np

MAGIC = b"RSXC"
VERSION = 1
_CODES = {np.dtype("<f4"): 0, np.dtype("<f8"): 1, np.dtype("<i4"): 2, np.dtype("<i8"): 3, np.dtype("<u2"): 4}
_DTYPES = {v: k for k, v in _CODES.items()}


def _host(a):
    try:
        import torch
        if isinstance(a, torch.Tensor):
            t = a.detach()
            if t.dtype == torch.bfloat16:
                t = t.view(torch.int16)
                return t.cpu().numpy().view(np.uint16)
            return t.cpu().numpy()
    except ImportError:
        pass
    return np.asarray(a)


def save(path, **arrays):
    """Write the named arrays to `path` (replacing it)."""
    with open(path, "wb") as f:
        for name, a in arrays.items():
            h = np.asarray(_host(a), order="C")
            dt = h.dtype.newbyteorder("<")
            if dt not in _CODES:
                raise ValueError(f"{name}: unsupported dtype {h.dtype}")
            h = h.astype(dt, copy=False)
            nb = name.encode("utf-8")
            f.write(MAGIC + struct.pack("<II", VERSION, len(nb)) + nb)
            f.write(struct.pack("<II", _CODES[dt], h.ndim))
            f.write(struct.pack(f"<{h.ndim}q", *h.shape))
            f.write(struct.pack("<Q", h.nbytes))
            f.write(h.tobytes(order="C"))


def load(path, device=None):
    """Read every record of `path`: {name: array} (torch tensors on `device` if given)."""
    out = {}
    with open(path, "rb") as f:
        data = f.read()
    pos = 0

    def take(n):
        nonlocal pos
        if pos + n > len(data):
            raise ValueError(f"{path}: truncated record at byte {pos}")
        b = data[pos:pos + n]
        pos += n
        return b

    while pos < len(data):
        if take(4) != MAGIC:
            raise ValueError(f"{path}: bad record magic at byte {pos - 4}")
        version, nlen = struct.unpack("<II", take(8))
        if version != VERSION:
            raise ValueError(f"{path}: unsupported record version {version}")
        name = take(nlen).decode("utf-8")
        code, ndim = struct.unpack("<II", take(8))
        if code not in _DTYPES:
            raise ValueError(f"{path}: {name}: unknown dtype code {code}")
        shape = struct.unpack(f"<{ndim}q", take(8 * ndim))
        (nbytes,) = struct.unpack("<Q", take(8))
        dt = _DTYPES[code]
        if nbytes != int(np.prod(shape, dtype=np.int64)) * dt.itemsize:
            raise ValueError(f"{path}: {name}: payload size {nbytes} does not match shape {shape}")
        arr = np.frombuffer(take(nbytes), dtype=dt).reshape(shape).copy()
        out[name] = arr
    if device is not None:
        import torch
        conv = {}
        for k, v in out.items():
            if v.dtype == np.uint16:
                conv[k] = torch.from_numpy(v.view(np.int16)).view(torch.bfloat16).to(device)
            else:
                conv[k] = torch.from_numpy(v).to(device)
        out = conv
    return out


# ---- stage helpers


def save_ground_state(path, orbitals, h, energies=None, xi=None):
    """Occupied orbitals [nocc][n^3-box], spacing, optional orbital energies and ACE projectors."""
    rec = {"orbitals": orbitals, "h": np.array([h], dtype=np.float64)}
    if energies is not None:
        rec["energies"] = np.asarray(_host(energies), dtype=np.float64)
    if xi is not None:
        rec["xi"] = xi
    save(path, **rec)


def save_casida(path, K, omega=None, X=None, Kd=None):
    """Coupling K (FP64 [nt][nt]), optional K_d, excitation energies and eigenvectors."""
    rec = {"K": K}
    for k, v in (("Kd", Kd), ("omega", omega), ("X", X)):
        if v is not None:
            rec[k] = v
    save(path, **rec)


def save_network(path, net, step=None):
    """The learned preconditioner's FP32 parameters (rsx_net_get_params) and the step
    count; the Adam moments stay in the network object, so a run resumed from this file
    restarts them from zero."""
    rec = {"params": np.asarray(net.get_params(), dtype=np.float32)}
    if step is not None:
        rec["step"] = np.array([step], dtype=np.int64)
    save(path, **rec)


def load_network(path, net):
    """Load parameters saved by save_network into `net` (rsx_net_set_params)."""
    rec = load(path)
    net.set_params(rec["params"])
    return rec
