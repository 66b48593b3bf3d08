"""rANS entropy coding of int16 residual codes: plain reference (test infrastructure).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: it shares no code with
the CUDA library.

The paper's TPC data, after track-model compression, go through rANS entropy
coding (Sec. 5; the asynchronous reconstruction times the TPC rANS decoding,
Table 2); it gives no format.  The coder here is range asymmetric numeral
systems as published by Duda (2013, "Asymmetric numeral systems: entropy
coding combining speed of Huffman coding with compression rate of arithmetic
coding"), with the parameters and layout below, which are this project's
format (the same one the CUDA library writes):

Symbols.  A code c in [-255, 255] is symbol c + 255; any other code (the
not-encoded marker -32768, clipped +-32767, large residuals) is the escape
symbol 511, and its raw value goes to an escape list.  Alphabet A = 512.

Model.  One static table per stream: the symbol counts n_s (total N) are
normalised to frequencies f_s summing to M = 2**12: f_s = max(1, n_s * M // N)
for n_s > 0, else 0; the excess D = M - sum(f) is then removed from (D < 0)
or added to (D > 0) the symbol with the largest frequency (ties: the lowest
symbol), by at most f - 1 per round when removing, until D = 0.  c_s is the
cumulative frequency of the symbols below s.

Coder.  32-bit state x in [L, 2**16 L), L = 2**16, 16-bit renormalisation.
Encoding symbol s: if x >= f_s * 2**(32 - 12), emit the word x mod 2**16 and
x //= 2**16; then x = (x // f_s) * M + (x mod f_s) + c_s.  Decoding: slot =
x mod M, s = the symbol with c_s <= slot < c_s + f_s, x = f_s * (x // M) +
slot - c_s; if x < L, x = x * 2**16 + the next word.

Layout.  The stream is cut into segments of S = 32 * T symbols (T = 512
steps); in a segment, symbol i belongs to lane i mod 32 at step i // 32, and
each of the 32 lanes is an independent rANS state starting at L.  Encoding
runs from the last step to the first; at each step the lanes that emit a word
(in increasing lane order) form a block, and the segment's words are the
blocks of steps 0, 1, ..., T-1 in that order -- exactly the order in which a
decoder running forward over the steps consumes them.  A segment's payload is
its 32 final states (uint32) followed by its words (uint16).

Container (little endian): 64-byte header (magic b"TPR1", version 1, n
symbols int64, segment symbols, segments, scale bits, alphabet uint32, escapes
int64, payload bytes int64, zero padding), frequency table (A x uint16),
segment byte offsets into the payload ((segments + 1) x uint64), segment
escape offsets ((segments + 1) x uint64), payload, escapes (int16).
"""
from __future__ import annotations

import struct

import numpy as np

ALPHABET = 512
ESCAPE = 511
CODE_RANGE = 255
SCALE_BITS = 12
M = 1 << SCALE_BITS
L = 1 << 16
LANES = 32
STEPS = 512
SEG = LANES * STEPS
MAGIC = b"TPR1"
HEADER_BYTES = 64


def symbols_of(codes: np.ndarray) -> np.ndarray:
    c = np.asarray(codes, dtype=np.int64)
    return np.where(np.abs(c) <= CODE_RANGE, c + CODE_RANGE, ESCAPE).astype(np.int64)


def normalise(counts: np.ndarray) -> np.ndarray:
    """Frequencies summing to M from symbol counts (the rule in the module doc)."""
    counts = np.asarray(counts, dtype=np.int64)
    n = int(counts.sum())
    f = np.zeros(ALPHABET, dtype=np.int64)
    if n == 0:
        return f
    for s in range(ALPHABET):
        if counts[s] > 0:
            f[s] = max(1, (int(counts[s]) * M) // n)
    d = M - int(f.sum())
    while d != 0:
        s = int(np.argmax(f))  # largest frequency, lowest symbol on ties
        if d > 0:
            f[s] += d
            d = 0
        else:
            take = min(-d, int(f[s]) - 1)
            f[s] -= take
            d += take
    return f


def _encode_segment(sym: np.ndarray, f: np.ndarray, cum: np.ndarray) -> tuple:
    n = len(sym)
    steps = (n + LANES - 1) // LANES
    x = [L] * LANES
    blocks = []  # blocks[k] = words emitted at step steps-1-k
    for step in range(steps - 1, -1, -1):
        block = []
        for lane in range(LANES):
            i = step * LANES + lane
            if i >= n:
                continue
            s = int(sym[i])
            fs, cs = int(f[s]), int(cum[s])
            if x[lane] >= fs << (32 - SCALE_BITS):
                block.append(x[lane] & 0xFFFF)
                x[lane] >>= 16
            x[lane] = (x[lane] // fs) * M + (x[lane] % fs) + cs
        blocks.append(block)
    words = [w for block in reversed(blocks) for w in block]
    return x, words


def encode(codes: np.ndarray, seg: int = SEG) -> bytes:
    """Encode int16 codes into the container described in the module doc."""
    codes = np.asarray(codes, dtype=np.int16)
    n = int(codes.shape[0])
    sym = symbols_of(codes)
    f = normalise(np.bincount(sym, minlength=ALPHABET))
    cum = np.concatenate([[0], np.cumsum(f)[:-1]])
    n_seg = (n + seg - 1) // seg
    payload, esc = bytearray(), []
    seg_off, esc_off = [0], [0]
    for j in range(n_seg):
        sl = slice(j * seg, min(n, (j + 1) * seg))
        states, words = _encode_segment(sym[sl], f, cum)
        payload += struct.pack("<32I", *states) + struct.pack("<%dH" % len(words), *words)
        seg_off.append(len(payload))
        esc += [int(v) for v, s in zip(codes[sl], sym[sl]) if s == ESCAPE]
        esc_off.append(len(esc))
    head = MAGIC + struct.pack("<IqIIIIqq", 1, n, seg, n_seg, SCALE_BITS, ALPHABET, len(esc), len(payload))
    head += b"\0" * (HEADER_BYTES - len(head))
    return (head + struct.pack("<%dH" % ALPHABET, *[int(v) for v in f]) +
            struct.pack("<%dQ" % (n_seg + 1), *seg_off) + struct.pack("<%dQ" % (n_seg + 1), *esc_off) +
            bytes(payload) + struct.pack("<%dh" % len(esc), *esc))


def parse(blob: bytes) -> dict:
    if blob[:4] != MAGIC:
        raise ValueError("not a TPR1 stream")
    ver, n, seg, n_seg, k, a, n_esc, n_pay = struct.unpack_from("<IqIIIIqq", blob, 4)
    if ver != 1 or k != SCALE_BITS or a != ALPHABET:
        raise ValueError("unsupported stream parameters")
    o = HEADER_BYTES
    f = np.frombuffer(blob, dtype="<u2", count=a, offset=o).astype(np.int64)
    o += 2 * a
    seg_off = np.frombuffer(blob, dtype="<u8", count=n_seg + 1, offset=o).astype(np.int64)
    o += 8 * (n_seg + 1)
    esc_off = np.frombuffer(blob, dtype="<u8", count=n_seg + 1, offset=o).astype(np.int64)
    o += 8 * (n_seg + 1)
    payload = blob[o:o + n_pay]
    o += n_pay
    esc = np.frombuffer(blob, dtype="<i2", count=n_esc, offset=o)
    return dict(n=n, seg=seg, n_seg=n_seg, f=f, seg_off=seg_off, esc_off=esc_off, payload=payload, esc=esc)


def decode(blob: bytes) -> np.ndarray:
    p = parse(blob)
    f = p["f"]
    cum = np.concatenate([[0], np.cumsum(f)[:-1]])
    slot_sym = np.repeat(np.arange(ALPHABET), f)  # M entries
    out = np.zeros(p["n"], dtype=np.int16)
    for j in range(p["n_seg"]):
        base, end = int(p["seg_off"][j]), int(p["seg_off"][j + 1])
        x = list(struct.unpack_from("<32I", p["payload"], base))
        words = struct.unpack_from("<%dH" % ((end - base - 128) // 2), p["payload"], base + 128)
        wi = 0
        ei = int(p["esc_off"][j])
        s0 = j * p["seg"]
        cnt = min(p["n"], s0 + p["seg"]) - s0
        for step in range((cnt + LANES - 1) // LANES):
            for lane in range(LANES):
                i = step * LANES + lane
                if i >= cnt:
                    continue
                slot = x[lane] & (M - 1)
                s = int(slot_sym[slot])
                x[lane] = int(f[s]) * (x[lane] >> SCALE_BITS) + slot - int(cum[s])
                if s == ESCAPE:
                    if ei >= int(p["esc_off"][j + 1]):
                        raise ValueError("segment %d reads past its escapes" % j)
                    out[s0 + i] = p["esc"][ei]
                    ei += 1
                else:
                    out[s0 + i] = s - CODE_RANGE
                if x[lane] < L:
                    if wi >= len(words):
                        raise ValueError("segment %d reads past its words" % j)
                    x[lane] = (x[lane] << 16) | words[wi]
                    wi += 1
        if wi != len(words) or ei != int(p["esc_off"][j + 1]) or any(v != L for v in x[:min(LANES, cnt)]):
            raise ValueError("segment %d does not decode to its initial states" % j)
    return out


def cross_entropy_bits(codes: np.ndarray) -> float:
    """Ideal size in bits of the codes under the normalised table."""
    sym = symbols_of(codes)
    cnt = np.bincount(sym, minlength=ALPHABET)
    f = normalise(cnt)
    nz = cnt > 0
    return float((cnt[nz] * np.log2(M / f[nz])).sum())
