"""rANS codec on the GPU against the reference coder (oracle/rans.py).

Integer work: the GPU container must equal the reference's byte for byte on
the same codes, and decode back to them.  At the full Pb-Pb size (two 192.6 M
code streams of the fitted frame's residuals) the reference is too slow for
the whole stream; there the frequency table, the offset tables and sampled
segments (re-encoded by the reference with the same table) are compared, and
the round trip is checked whole.
"""
import struct
import types

import numpy as np
import pytest

import tpcgen
from oracle import rans

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_01205_gb300 as T
    from paper_2402_01205_gb300 import _build
    _build.build()
    return T


def gpu_encode(T, fx, codes, seg=0):
    d = torch.from_numpy(np.ascontiguousarray(codes, dtype=np.int16)).cuda()
    out, size = fx.rans_encode(d, segment_symbols=seg)
    return out, size, bytes(out[:size].cpu().numpy().tobytes())


@pytest.mark.parametrize("n,seg", [(0, 0), (1, 0), (33, 128), (1000, 128), (70_001, 4096), (100_000, 0)])
def test_bytes_equal_reference_and_round_trip(T, n, seg):
    rng = np.random.default_rng(n)
    c = np.round(rng.normal(0, 15, n)).astype(np.int16)
    c[rng.random(n) < 0.01] = -32768
    c[rng.random(n) < 0.002] = 30000
    with T.Fitter() as fx:
        out, size, blob = gpu_encode(T, fx, c, seg)
        ref = rans.encode(c, seg=seg or rans.SEG)
        assert blob == ref
        back = fx.rans_decode(out, size, n)
        assert np.array_equal(back.cpu().numpy(), c)
        assert np.array_equal(rans.decode(blob), c)


def test_single_symbol_and_all_escapes(T):
    with T.Fitter() as fx:
        for c in (np.full(50_000, -3, np.int16), np.full(9_999, -32768, np.int16)):
            out, size, blob = gpu_encode(T, fx, c, 1024)
            assert blob == rans.encode(c, seg=1024)
            assert np.array_equal(fx.rans_decode(out, size, len(c)).cpu().numpy(), c)


def test_residual_codes_of_a_fit(T):
    f = tpcgen.generate("detector50k", n_tracks=20_000, seed=13)
    g = types.SimpleNamespace(**{k: torch.from_numpy(np.ascontiguousarray(getattr(f, k))).cuda()
                                 for k in ("offsets", "x", "y", "z", "sy2", "sz2", "row")})
    with T.Fitter() as fx:
        res = fx.fit(g, T.alloc_result(f.n_tracks, f.n_clusters, device="cuda", residuals=True))
        for k in ("res_y", "res_z"):
            out, size = fx.rans_encode(res[k])
            blob = bytes(out[:size].cpu().numpy().tobytes())
            assert blob == rans.encode(res[k].cpu().numpy())
            assert torch.equal(fx.rans_decode(out, size, f.n_clusters), res[k])
            print(k, "bits per code %.3f" % (8 * size / f.n_clusters))


def test_full_size_pbpb_residuals_sampled(T):
    f = tpcgen.generate("pbpb2m")
    g = types.SimpleNamespace(**{k: torch.from_numpy(np.ascontiguousarray(getattr(f, k))).cuda()
                                 for k in ("offsets", "x", "y", "z", "sy2", "sz2", "row")})
    with T.Fitter() as fx:
        res = fx.fit(g, T.alloc_result(f.n_tracks, f.n_clusters, device="cuda", residuals=True))
        del g
        codes = res["res_y"]
        out, size = fx.rans_encode(codes)
        host = out[:size].cpu().numpy().tobytes()
        p = rans.parse(host)
        cnp = codes.cpu().numpy()
        sym = rans.symbols_of(cnp)
        assert np.array_equal(p["f"], rans.normalise(np.bincount(sym, minlength=rans.ALPHABET)))
        assert p["n"] == f.n_clusters and p["n_seg"] == -(-f.n_clusters // rans.SEG)
        cum = np.concatenate([[0], np.cumsum(p["f"])[:-1]])
        for j in np.linspace(0, p["n_seg"] - 1, 12).astype(int):
            sl = slice(j * rans.SEG, min(len(cnp), (j + 1) * rans.SEG))
            states, words = rans._encode_segment(sym[sl], p["f"], cum)
            want = struct.pack("<32I", *states) + struct.pack("<%dH" % len(words), *words)
            assert p["payload"][p["seg_off"][j]:p["seg_off"][j + 1]] == want, j
            esc = [int(v) for v, s in zip(cnp[sl], sym[sl]) if s == rans.ESCAPE]
            assert list(p["esc"][p["esc_off"][j]:p["esc_off"][j + 1]]) == esc
        back = fx.rans_decode(out, size, f.n_clusters)
        assert torch.equal(back, codes)
        print("bits per code %.3f, cross-entropy %.3f" % (8 * size / len(cnp), rans.cross_entropy_bits(cnp) / len(cnp)))


def test_damaged_or_mismatched_streams_are_rejected(T):
    rng = np.random.default_rng(7)
    c = np.round(rng.normal(0, 12, 50_000)).astype(np.int16)
    with T.Fitter() as fx:
        out, size, blob = gpu_encode(T, fx, c, 2048)
        with pytest.raises(T.TpcfitError) as ei:
            fx.rans_decode(out, size, len(c) + 1)  # wrong count
        assert ei.value.code == T.E_INVAL
        with pytest.raises(T.TpcfitError):
            fx.rans_decode(out, size - 2, len(c))  # truncated
        p = rans.parse(blob)
        pay0 = len(blob) - 2 * len(p["esc"]) - len(p["payload"])
        for off in (pay0 + 128 + 100, pay0 + 5, 64 + 2 * 255):  # a word, a state, the frequency table
            bad = bytearray(blob)
            bad[off] ^= 0xA5
            d = torch.from_numpy(np.frombuffer(bytes(bad), np.uint8).copy()).cuda()
            try:
                r = fx.rans_decode(d, size, len(c)).cpu().numpy()
            except T.TpcfitError as e:
                assert e.code == T.E_INVAL
                continue
            assert not np.array_equal(r, c), off
        # the handle stays usable
        assert np.array_equal(fx.rans_decode(out, size, len(c)).cpu().numpy(), c)
