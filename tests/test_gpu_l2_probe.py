"""The L2 read-bandwidth probe (sc_l2_read) reads every word: with an odd
number of passes the XOR of the blocks' sinks equals the XOR of the
buffer's 32-bit words; bad arguments are refused before any launch."""
import numpy as np
import pytest

from paper_2305_08343_gb300 import subcull as sc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_probe_reads_every_word_and_checks_arguments():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    nb = sc.sc_l2_probe_blocks()
    assert nb > 0
    words = np.random.default_rng(3).integers(0, 2 ** 32, (1 << 20) + 4, dtype=np.uint32)
    buf = torch.from_numpy(words.view(np.int32)).cuda()
    sink = torch.zeros(nb, dtype=torch.int64, device="cuda")
    sc.sc_l2_read(buf, 3, sink)
    torch.cuda.synchronize()
    folded = np.bitwise_xor.reduce(sink.cpu().numpy().astype(np.uint64))
    assert int(folded) == int(np.bitwise_xor.reduce(words))
    with pytest.raises(sc.SubcullError):
        sc.sc_l2_read(buf[1:], 1, sink)  # 4-byte offset: misaligned
    with pytest.raises(sc.SubcullError):
        sc.sc_l2_read(buf, 0, sink)
