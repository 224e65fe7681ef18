"""Surrogate checkpoints: the file format round-trips parameters and Adam
state exactly, the parameter count matches the library's layout, and damaged
files are rejected (host-side only, no GPU)."""
import numpy as np
import pytest

from paper_2006_06743_gb300 import datagen
from paper_2006_06743_gb300 import surrogate as sg


def test_counts_match_the_library_layout():
    sng = pytest.importorskip("paper_2006_06743_gb300")
    try:
        sng.lib()
    except Exception:
        pytest.skip("libsng.so not built")
    for d in (1, 3, 32, 64):
        assert sg._counts(d)[0] == sg.param_count(d)
        assert sg._counts(d)[1] == sg.trained_count(d)


@pytest.mark.parametrize("moments", [False, True])
def test_round_trip(tmp_path, moments):
    d = 7
    init = datagen.mlp_init(d, sg.HIDDEN, 3)
    rng = np.random.default_rng(0)
    mean, std = rng.normal(size=d), rng.uniform(0.5, 2.0, size=d)
    vec = np.concatenate([np.asarray(init[k], np.float32).ravel()
                          for k in ("w1", "b1", "w2", "b2", "w3", "b3")]
                         + [mean.astype(np.float32), std.astype(np.float32)])
    nt = sg._counts(d)[1]
    m = rng.normal(size=nt).astype(np.float32) if moments else None
    v = rng.uniform(size=nt).astype(np.float32) if moments else None
    path = str(tmp_path / "net.bin")
    sg.save_params(path, vec, d, step=123, m=m, v=v)
    ck = sg.load_params(path)
    assert ck["d"] == d and ck["step"] == 123
    np.testing.assert_array_equal(ck["params"], vec)
    if moments:
        np.testing.assert_array_equal(ck["m"], m)
        np.testing.assert_array_equal(ck["v"], v)
    else:
        assert ck["m"] is None and ck["v"] is None


def test_damaged_files_are_rejected(tmp_path):
    d = 4
    vec = np.zeros(sg._counts(d)[0], np.float32)
    path = tmp_path / "net.bin"
    sg.save_params(str(path), vec, d)
    blob = path.read_bytes()
    bad = tmp_path / "bad.bin"
    for damaged in (b"XXXXXXXX" + blob[8:], blob[:-4], blob + b"\0\0\0\0", blob[:20]):
        bad.write_bytes(damaged)
        with pytest.raises(ValueError):
            sg.load_params(str(bad))
    with pytest.raises(ValueError):
        sg.save_params(str(bad), vec[:-1], d)
