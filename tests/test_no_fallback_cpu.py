"""The product path has no CPU fallback: without its CUDA library, or
without a CUDA device, it fails loudly instead of computing anything."""
import pytest

torch = pytest.importorskip("torch")

from paper_1712_09430_gb300 import build_ext, capi, synth  # noqa: E402
from paper_1712_09430_gb300.tracker import Tracker, TrackerError  # noqa: E402


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(capi, "_LIB", None)
    monkeypatch.setattr(build_ext, "LIB", str(tmp_path / "libtpcca.so"))
    monkeypatch.setattr(build_ext, "up_to_date", lambda: True)
    with pytest.raises(RuntimeError, match="library missing"):
        capi.lib()


def test_failed_build_raises(monkeypatch, tmp_path):
    def fail():
        raise RuntimeError("nvcc failed")
    monkeypatch.setattr(capi, "_LIB", None)
    monkeypatch.setattr(build_ext, "LIB", str(tmp_path / "libtpcca.so"))
    monkeypatch.setattr(build_ext, "up_to_date", lambda: False)
    monkeypatch.setattr(build_ext, "build", fail)
    with pytest.raises(RuntimeError, match="nvcc failed"):
        capi.lib()


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a CUDA device")
def test_no_device_is_an_error_not_a_cpu_run():
    with pytest.raises(TrackerError, match="TPC_ERR_DEVICE"):
        Tracker(synth.row_x(), bz=0.5)


def test_unknown_parameter_name_is_an_error():
    from paper_1712_09430_gb300.tracker import default_params
    p = default_params(bin_target=0.5, field=(1e-5, 0, 0, 0, 0))
    assert p.bin_target == 0.5 and abs(p.field[0] - 1e-5) < 1e-12
    with pytest.raises(TypeError, match="unknown tracker parameter"):
        default_params(bin_targt=0.5)
