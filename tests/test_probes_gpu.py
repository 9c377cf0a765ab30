"""The bandwidth probes on the GPU: the STREAM triad writes a = b + s*c (inputs
chosen so that the fused multiply-add and the separate product and sum agree
exactly), and the read probe touches every 16-byte word of its buffer."""
import pytest

from paper_2606_22423_gb300 import gbscan

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.init()
    return gbscan.load()


@pytest.mark.parametrize("n", [0, 4, 1 << 12, (1 << 20) + 4, (3 << 22) + 12])
def test_triad_is_exact(n):
    g = torch.Generator(device="cpu").manual_seed(n)
    b = torch.randint(-1024, 1024, (n,), generator=g).float().cuda()
    c = torch.randint(-1024, 1024, (n,), generator=g).float().cuda()
    a = torch.full((n,), float("nan"), device="cuda")
    s = torch.cuda.Stream()
    gbscan.scan_probe_triad(a, b, c, 3.0, n, s)
    s.synchronize()
    assert torch.equal(a, b + 3.0 * c)


def test_read_probe_sees_every_word():
    """Every word of the buffer is read: a buffer whose words xor to zero in
    every 16-byte group except one gives a checksum that depends on that group."""
    n16 = (1 << 20) + 3
    buf = torch.zeros(n16 * 4, dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    gbscan.scan_probe_read(buf, n16 * 16, out, s)
    s.synchronize()
    assert int(out.item()) == 0
    buf[4 * (n16 - 1)] = 5          # the last 16-byte group
    gbscan.scan_probe_read(buf, n16 * 16, out, s)
    s.synchronize()
    assert int(out.item()) == 5
