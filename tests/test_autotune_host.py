"""Autotuner cache key (host only): a choice is keyed by the batch shape, the
device and the built library, so a rebuild or another GPU times again."""
from paper_2601_20758_gb300 import _lib as L
from paper_2601_20758_gb300 import autotune


def test_signature_holds_shape_device_and_build(tmp_path):
    p = L.make_params(rule=L.SF_BW_KNN, k=64)
    dims = [(64, 64, 64), (32, 32, 32)]
    a = autotune.signature(1 << 20, dims, L.SF_K_GAUSS3, p, "GPU-A-sm103", "abc")
    assert a == autotune.signature(1 << 20, dims, L.SF_K_GAUSS3, p, "GPU-A-sm103", "abc")
    assert a != autotune.signature(1 << 20, dims, L.SF_K_GAUSS3, p, "GPU-B-sm100", "abc")
    assert a != autotune.signature(1 << 20, dims, L.SF_K_GAUSS3, p, "GPU-A-sm103", "abd")
    assert a != autotune.signature(1 << 20, dims, L.SF_K_EPAN, p, "GPU-A-sm103", "abc")
    q = L.make_params(rule=L.SF_BW_KNN, k=64)
    q.prec = L.SF_PREC_BF16
    assert a != autotune.signature(1 << 20, dims, L.SF_K_GAUSS3, q, "GPU-A-sm103", "abc")


def test_library_digest_follows_the_file(tmp_path):
    f = tmp_path / "lib.so"
    f.write_bytes(b"one build")
    d1 = autotune.library_digest(str(f))
    assert len(d1) == 12 and d1 == autotune.library_digest(str(f))
    f.write_bytes(b"another build, longer")
    assert autotune.library_digest(str(f)) != d1
