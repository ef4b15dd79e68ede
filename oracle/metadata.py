"""Packed split metadata (Sec. 4.3, Tables 1-2) -- TEST INFRASTRUCTURE ONLY.

Plain Python restatement of the paper's metadata storage, bit by bit, used to
check the library's serialiser. Readings (the paper's prose, not its code):

* Header: M (splits, counting the final-state one), B (bitstream length in
  16-bit words) and N (symbols), stored as-is in 32, 64 and 64 bits.
* Split point i = 1 .. M-1 (the regular entries in order): its word offset q_i
  (0-based index of the split word) is stored as q_i - i * ceil(B / M), and its
  anchor (the largest group ID of its coders) as anchor_i - i * ceil(G / M),
  G = ceil(N / W). These two signed series cover all split points (Table 1).
* Group IDs are 1-based, ceil(i / W) for a 1-based symbol index (Table 2), i.e.
  idx // W + 1 for our 0-based recorded index idx.
* Per split point: the W states as-is (16 bits each, Lemma 3.1), then the
  series of anchor - group ID, all >= 0, stored without sign (Table 2).
* A series is a width field holding (w - 1) followed by every value in w bits,
  w = the bit length of the largest magnitude (1 when all are zero). The
  paper's count floor(log2(v + 1)) is one short for v = 2, 6, 14, ...; the bit
  length is the count that always fits. Unsigned series (group-ID
  differences, up to 16 bits) use a 4-bit width field; signed series (up to 32
  bits) a 5-bit field and one sign bit before each magnitude.
* Bits are written most significant first; the section is padded with zero
  bits to whole bytes.
"""
from __future__ import annotations

import math

W = 32


class BitWriter:
    def __init__(self):
        self.bits: list[int] = []

    def put(self, value: int, width: int):
        for k in range(width - 1, -1, -1):
            self.bits.append((value >> k) & 1)

    def to_bytes(self) -> bytes:
        bits = self.bits + [0] * (-len(self.bits) % 8)
        return bytes(int("".join(map(str, bits[i:i + 8])), 2) for i in range(0, len(bits), 8))


class BitReader:
    def __init__(self, data: bytes):
        self.bits = [(byte >> (7 - k)) & 1 for byte in data for k in range(8)]
        self.pos = 0

    def get(self, width: int) -> int:
        v = 0
        for _ in range(width):
            v = (v << 1) | self.bits[self.pos]
            self.pos += 1
        return v


def bit_length(v: int) -> int:
    return max(1, int(v).bit_length())


def put_unsigned_series(bw: BitWriter, values, field_bits: int = 4):
    w = max([bit_length(v) for v in values] + [1])
    if w > (1 << field_bits):
        raise ValueError("value too wide for its series")
    bw.put(w - 1, field_bits)
    for v in values:
        bw.put(int(v), w)


def put_signed_series(bw: BitWriter, values, field_bits: int = 5):
    w = max([bit_length(abs(v)) for v in values] + [1])
    if w > (1 << field_bits):
        raise ValueError("value too wide for its series")
    bw.put(w - 1, field_bits)
    for v in values:
        bw.put(1 if v < 0 else 0, 1)
        bw.put(abs(int(v)), w)


def get_unsigned_series(br: BitReader, count: int, field_bits: int = 4):
    w = br.get(field_bits) + 1
    return [br.get(w) for _ in range(count)]


def get_signed_series(br: BitReader, count: int, field_bits: int = 5):
    w = br.get(field_bits) + 1
    out = []
    for _ in range(count):
        neg = br.get(1)
        mag = br.get(w)
        out.append(-mag if neg else mag)
    return out


def pack(M: int, B: int, N: int, q, idx, y, W: int = W) -> bytes:
    """Metadata of M splits; q[i], idx[i][j], y[i][j] for the M-1 regular entries in order.

    W (coders) is 32 for every stream the library makes; the worked example of
    Tables 1-2 has 4."""
    bw = BitWriter()
    bw.put(M, 32)
    bw.put(B, 64)
    bw.put(N, 64)
    Eb = math.ceil(B / M) if M else 0
    G = math.ceil(N / W)
    Eg = math.ceil(G / M) if M else 0
    anchors = [max(int(v) // W + 1 for v in row) for row in idx]
    put_signed_series(bw, [int(q[i]) - (i + 1) * Eb for i in range(M - 1)])
    put_signed_series(bw, [anchors[i] - (i + 1) * Eg for i in range(M - 1)])
    for i in range(M - 1):
        for j in range(W):
            bw.put(int(y[i][j]), 16)
        put_unsigned_series(bw, [anchors[i] - (int(idx[i][j]) // W + 1) for j in range(W)])
    return bw.to_bytes()


def unpack(data: bytes, W: int = W):
    """Inverse of pack: (M, B, N, q, idx, y)."""
    br = BitReader(data)
    M = br.get(32)
    B = br.get(64)
    N = br.get(64)
    Eb = math.ceil(B / M) if M else 0
    G = math.ceil(N / W)
    Eg = math.ceil(G / M) if M else 0
    dq = get_signed_series(br, M - 1)
    da = get_signed_series(br, M - 1)
    q, idx, y = [], [], []
    for i in range(M - 1):
        q.append((i + 1) * Eb + dq[i])
        anchor = (i + 1) * Eg + da[i]
        states = [br.get(16) for _ in range(W)]
        diffs = get_unsigned_series(br, W)
        y.append(states)
        idx.append([(anchor - diffs[j] - 1) * W + j for j in range(W)])
    return M, B, N, q, idx, y
