"""The network checkpoint format on the CPU: files written here by an independent Python writer
(struct + zlib's CRC-32) following the layout that include/elrt.h documents are accepted by the
library's validator with the right description; damaged files are rejected."""

import os
import struct
import zlib

import numpy as np
import pytest


def _layout(p, n_angles, n_hidden, width):
    n1 = p + 1
    nm, nin = n1 * n1, 2 * n1 * n_angles
    fpad = (nm + 1 + 63) // 64 * 64
    nout = nin * nin + nm * nin
    sizes = []
    for l in range(n_hidden + 1):
        in_pad = fpad if l == 0 else width
        out = nout if l == n_hidden else width
        sizes += [out * in_pad, out, out * in_pad, out * in_pad, out, out]
    return sizes + [fpad, fpad, nout, nout]


def _write(path, p=2, n_angles=4, n_hidden=1, width=64, act=1, seed=99, standardised=1, step=17, count=None,
           features=1):
    n = sum(_layout(p, n_angles, n_hidden, width)) if count is None else count
    head = b"ELRTNET\0" + struct.pack("<IiiiiiQiqqi", 2, p, n_angles, n_hidden, width, act, seed, standardised, step, n,
                                       features)
    assert len(head) == 64
    vals = np.random.default_rng(0).normal(size=n).astype("<f4").tobytes()
    body = head + vals
    with open(path, "wb") as f:
        f.write(body + struct.pack("<I", zlib.crc32(body) & 0xFFFFFFFF))
    return n


@pytest.fixture
def E():
    import paper_2308_02467_gb300 as E
    return E


def test_valid_file_is_read(E, tmp_path):
    path = str(tmp_path / "net.bin")
    n = _write(path)
    info = E.elrt_net_file_info(path)
    assert info == {"p": 2, "n_angles": 4, "n_hidden": 1, "width": 64, "activation": 1, "seed": 99, "features": 1,
                    "standardised": 1, "adam_step": 17, "n_values": n}


@pytest.mark.parametrize("damage", ["flip", "truncate", "append", "count", "magic", "version", "desc", "features"])
def test_damaged_file_is_rejected(E, tmp_path, damage):
    path = str(tmp_path / "net.bin")
    if damage == "count":
        _write(path, count=sum(_layout(2, 4, 1, 64)) - 1)
    elif damage == "desc":
        _write(path, n_angles=6)                       # N not a multiple of 4
    elif damage == "features":
        _write(path, features=2)
    else:
        _write(path)
        b = bytearray(open(path, "rb").read())
        if damage == "flip":
            b[100] ^= 0x10
        elif damage == "truncate":
            b = b[:-9]
        elif damage == "append":
            b += b"\0"
        elif damage == "magic":
            b[0] = ord("X")
        elif damage == "version":
            b[8] = 1
        open(path, "wb").write(bytes(b))
    with pytest.raises(E.ElrtError) as ei:
        E.elrt_net_file_info(path)
    assert ei.value.status == 1


def test_missing_file_is_rejected(E, tmp_path):
    with pytest.raises(E.ElrtError):
        E.elrt_net_file_info(str(tmp_path / "absent.bin"))
