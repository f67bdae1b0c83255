"""The gather-bandwidth probe (a measurement utility): it must read exactly the rows it is
given.  The XOR of every thread's sink equals the XOR of all 32-bit words of the gathered
rows (rows read an even number of times cancel), plus row 0 once per padding slot of the
last 32-index chunk."""
import numpy as np
import pytest

from _util import dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_2604_27985_gb300 as g

    return g


def _expected(table_u32, idx, row_words):
    rx = np.bitwise_xor.reduce(table_u32[:, :row_words], axis=1)
    pad = (-len(idx)) % 32
    acc = np.bitwise_xor.reduce(rx[idx]) if len(idx) else np.uint32(0)
    if pad % 2:
        acc ^= rx[0]
    return np.uint32(acc)


@pytest.mark.parametrize("row_bytes,ld_words", [(128, 32), (256, 64), (512, 128), (256, 72), (1024, 256), (1024, 264)])
@pytest.mark.parametrize("unroll", [4, 8])
@pytest.mark.parametrize("n", [1, 31, 32, 1000, 100003])
def test_probe_reads_every_row(gb, row_bytes, ld_words, unroll, n):
    import torch

    rng = np.random.default_rng(n + row_bytes)
    rows = 3000
    table = rng.integers(0, 2**32, size=(rows, ld_words), dtype=np.uint64).astype(np.uint32)
    idx = rng.integers(0, rows, size=n).astype(np.int32)
    t = dev(table.view(np.int32))
    blocks = 7
    sink = torch.zeros(blocks * 256, dtype=torch.int32, device="cuda")
    gb.gather_probe(t, dev(idx), row_bytes, blocks=blocks, unroll=unroll, sink=sink)
    got = np.bitwise_xor.reduce(sink.cpu().numpy().view(np.uint32))
    assert got == _expected(table, idx, row_bytes // 4)


def test_probe_argument_errors(gb):
    import torch

    t = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    idx = torch.zeros(10, dtype=torch.int32, device="cuda")
    with pytest.raises(gb.GbspError, match="UNSUPPORTED"):
        gb.gather_probe(t, idx, 100)
    with pytest.raises(gb.GbspError, match="ALIGN"):
        gb.gather_probe(t.view(-1)[1:4033].view(63, 64), idx, 128)
