"""Helpers for the persistence tests: the documented file checksum, written
independently of the library (test helper)."""
import struct

MASK = (1 << 64) - 1
HEADER_BYTES = 1024
O_VERSION, O_FANOUT, O_LEVELS, O_NODES = 8, 16, 28, 40
O_LEVEL_NODES = 64
O_PAYLOAD_BYTES = O_LEVEL_NODES + 8 * 40
O_PAYLOAD_HASH = O_PAYLOAD_BYTES + 8
O_HEADER_HASH = O_PAYLOAD_HASH + 8


def file_hash(data: bytes) -> int:
    """64-bit words, little-endian, tail zero-padded: h = rotl(h, 27) ^ w,
    h *= 0x9E3779B97F4A7C15, from 0x243F6A8885A308D3; then h ^ length."""
    n = len(data)
    padded = data + b"\0" * (-n % 8)
    h = 0x243F6A8885A308D3
    for (w,) in struct.iter_unpack("<Q", padded):
        h = ((h << 27) | (h >> 37)) & MASK
        h = ((h ^ w) * 0x9E3779B97F4A7C15) & MASK
    return h ^ n


def reseal(buf: bytearray) -> bytearray:
    """Recomputes the payload and header checksums of a tree file image."""
    payload = bytes(buf[HEADER_BYTES:])
    struct.pack_into("<Q", buf, O_PAYLOAD_HASH, file_hash(payload))
    struct.pack_into("<Q", buf, O_HEADER_HASH, 0)
    struct.pack_into("<Q", buf, O_HEADER_HASH, file_hash(bytes(buf[:HEADER_BYTES])))
    return buf
