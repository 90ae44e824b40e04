"""Stream checkpoint blobs, checked on the host without a GPU: a blob built here from the
layout documented in include/frr.h is accepted and described field by field; a flipped
byte, a truncated or padded blob, a wrong magic or a retained count that does not match the
size are rejected with FRR_E_ARG, and an unknown version with FRR_E_UNSUPPORTED."""
import struct

import numpy as np
import pytest

FNV_OFFSET, FNV_PRIME = 0xCBF29CE484222325, 0x100000001B3


@pytest.fixture(scope="module")
def frr():
    from paper_2501_07642_b300 import build
    build.build_library()
    from paper_2501_07642_b300 import frr as f
    return f


def _fnv1a(data: bytes) -> int:
    h = FNV_OFFSET
    for b in data:
        h = ((h ^ b) * FNV_PRIME) & 0xFFFFFFFFFFFFFFFF
    return h


def _blob(r=5, version=1, magic=b"FRRSTRM\0", seen=3_000_000, total=100_000_000):
    idx = np.arange(r, dtype="<u8") * 7919 + 11
    mh = np.linspace(1.0, 2.0, r, dtype="<f4")
    hdr = bytearray(256)
    hdr[0:8] = magic
    struct.pack_into("<II", hdr, 8, version, 256)
    struct.pack_into("<qqq", hdr, 16, 1000, 1000, 500)
    struct.pack_into("<ii", hdr, 40, 0, 1)
    struct.pack_into("<dd", hdr, 48, 0.1, 2.0)
    struct.pack_into("<ddd", hdr, 64, 1e-3, 1e-6, 1e-7)
    struct.pack_into("<QQQ", hdr, 88, 5, total, seen)
    struct.pack_into("<ii", hdr, 112, 0, 1)
    struct.pack_into("<dd", hdr, 120, 1.2e-5, float("nan"))
    struct.pack_into("<qq", hdr, 136, 1200, r)
    struct.pack_into("<f", hdr, 152, 800.5)
    struct.pack_into("<qdd", hdr, 160, seen, 9.0, 0.5)
    body = bytes(hdr) + idx.tobytes() + mh.tobytes()
    ck = _fnv1a(body)  # the checksum field (bytes 248-255) is zero here
    out = bytearray(body)
    struct.pack_into("<Q", out, 248, ck)
    return bytes(out)


def test_blob_info_reads_the_documented_layout(frr):
    info = frr.frr_stream_blob_info(_blob())
    assert info["version"] == 1 and (info["n"], info["d"], info["n1"]) == (1000, 1000, 500)
    assert (info["seed"], info["total"], info["seen"]) == (5, 100_000_000, 3_000_000)
    assert info["q"] == 1.2e-5 and np.isnan(info["threshold"])
    assert (info["K"], info["retained"]) == (1200, 5)
    assert frr.frr_stream_blob_info(_blob(r=0))["retained"] == 0


@pytest.mark.parametrize("damage", ["flip_header", "flip_payload", "truncate", "pad", "magic", "count", "seen"])
def test_damaged_blobs_are_rejected(frr, damage):
    b = bytearray(_blob())
    if damage == "flip_header":
        b[100] ^= 0x01
    elif damage == "flip_payload":
        b[-3] ^= 0x40
    elif damage == "truncate":
        b = b[:-1]
    elif damage == "pad":
        b = b + b"\0" * 12
    elif damage == "magic":
        b = bytearray(_blob(magic=b"FRRSTRX\0"))
    elif damage == "count":
        struct.pack_into("<q", b, 144, 6)  # one more pair than the blob holds (checksum now wrong too)
    elif damage == "seen":
        b = bytearray(_blob(seen=200, total=100))
    with pytest.raises(frr.FrrError) as e:
        frr.frr_stream_blob_info(bytes(b))
    assert e.value.name == "FRR_E_ARG"


def test_unknown_version_is_unsupported(frr):
    with pytest.raises(frr.FrrError) as e:
        frr.frr_stream_blob_info(_blob(version=2))
    assert e.value.name == "FRR_E_UNSUPPORTED"
