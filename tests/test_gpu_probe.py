"""The streaming-read probe behind the benchmark's L2 figure reads every
byte it is given: over a buffer of ones, `passes` reads sum to exactly
passes x floats (all partial sums are small integers); sizes that are not a
multiple of 16 bytes are rejected before any launch."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_probe_reads_every_float():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_04403_gb300 import build as B
    B.build()
    import paper_2305_04403_gb300 as wob
    buf = torch.ones(1 << 20, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float32, device="cuda")
    wob.probe_l2_read(buf, 3, out)
    assert out.item() == 3.0 * (1 << 20)
    with pytest.raises(wob.WobError):
        wob.probe_l2_read(buf[:3], 1, out)
