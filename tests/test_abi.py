"""C-ABI library: builds, loads and exports every declared entry point (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            src = open(os.path.join(inc, fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(tpcfit_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2402_01205_gb300 import _build
    _build.build()
    return ctypes.CDLL(_build.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"tpcfit_create", "tpcfit_fit", "tpcfit_submit", "tpcfit_poll", "tpcfit_destroy"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_default_config_and_errors_without_gpu(lib):
    import paper_2402_01205_gb300 as T
    cfg = T.default_config()
    assert cfg.bz_tesla == pytest.approx(0.5) and cfg.chi2_max == 16.0 and cfg.min_clusters == 10
    assert cfg.n_rows == 152 and cfg.restart_scale == 100.0 and cfg.sort_tracks == 1
    assert list(cfg.seed_cov) == pytest.approx([1, 1, 0.01, 0.01, 1])
    assert T.strerror(T.E_NODEV).startswith("no usable CUDA device")
    import torch
    if not torch.cuda.is_available():
        with pytest.raises(T.TpcfitError) as ei:
            T.create(cfg)
        assert ei.value.code == T.E_NODEV
    bad = T.default_config(n_rows=300)
    with pytest.raises(T.TpcfitError) as ei:
        T.create(bad)
    assert ei.value.code == T.E_INVAL


def test_struct_layout_matches_header(lib, tmp_path):
    """ctypes mirrors of the C structs have the C compiler's offsets and sizes."""
    import subprocess
    import paper_2402_01205_gb300 as T
    structs = {"tpcfit_config": T.Config, "tpcfit_frame": T._Frame, "tpcfit_result": T._Result,
               "tpcfit_timing": T._Timing, "tpcfit_follow_config": T.FollowConfig, "tpcfit_hits": T._Hits,
               "tpcfit_seeds": T._Seeds, "tpcfit_tracks": T._Tracks}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tpcfit.h"', '#include "tpcfit_follow.h"',
             "int main(void){"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split("\n")
    got = {}
    for ln in out:
        if ln:
            c, f, v = ln.split()
            got[(c, f)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_binding_declares_the_signature_of_every_entry_point():
    """ctypes passes undeclared arguments as C int: a pointer or an int64_t
    would be truncated.  The binding must declare every entry point it can call."""
    import paper_2402_01205_gb300 as T
    lib = T._load()
    missing = [n for n in sorted(_declared()) if getattr(lib, n).argtypes is None]
    assert not missing, missing
    for n in ("tpcfit_rans_bound", "tpcfit_now"):
        assert getattr(lib, n).restype in (ctypes.c_int64, ctypes.c_double), n


def test_binding_marshals_host_frames_without_x():
    """A host frame may leave x out (clusters on their pad-row planes): the C
    frame then carries a NULL x and the cluster count of y; other arrays are
    required."""
    import types

    import numpy as np

    import paper_2402_01205_gb300 as T
    import tpcgen
    f = tpcgen.generate("sector1k", n_tracks=12)
    arrays = {k: np.ascontiguousarray(getattr(f, k)) for k in ("y", "z", "sy2", "sz2", "row")}
    c, mem, nt, nc = T._frame_struct(types.SimpleNamespace(offsets=f.offsets, x=None, **arrays))
    assert c.x is None and c.y and mem == T.MEM_HOST and (nt, nc) == (f.n_tracks, f.n_clusters)
    full, *_ = T._frame_struct(f)
    assert full.x and full.n_clusters == c.n_clusters
    bad = dict(arrays, z=None)
    with pytest.raises(ValueError):
        T._frame_struct(types.SimpleNamespace(offsets=f.offsets, x=None, **bad))


def test_results_of_another_frame_are_rejected_before_any_launch():
    """Every result buffer is checked against the frame it is for (state and
    cov per track, accept and residual codes per cluster): a result sized for
    a smaller frame raises ValueError in the binding, so no kernel or copy
    ever writes past it.  Handle 0 is never reached."""
    import numpy as np

    import paper_2402_01205_gb300 as T
    import tpcgen
    f = tpcgen.generate("sector1k", n_tracks=40)
    small = tpcgen.generate("sector1k", n_tracks=39)
    good = T.alloc_result(f.n_tracks, f.n_clusters, residuals=True)
    T._result_struct(good, f.n_tracks, f.n_clusters)  # the right sizes pass
    for k in ("state", "cov", "chi2", "status", "accept", "res_y"):
        res = dict(good)
        res[k] = T.alloc_result(small.n_tracks, small.n_clusters, residuals=True)[k]
        for call in (lambda: T.fit(0, f, res), lambda: T.submit(0, f, res), lambda: T.fit_noalloc(f, res)):
            with pytest.raises(ValueError, match=k):
                call()
    res = dict(good, restart_state=np.empty((f.n_tracks - 1, 5), np.float32))
    with pytest.raises(ValueError, match="restart_state"):
        T.fit(0, f, res)
