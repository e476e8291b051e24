"""The instruction-throughput probe computes what its declaration says
(host emulation of every chain for a few iterations), times every CTA, and
rejects unknown operations and CTA counts that cannot be resident."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1101_1427_gb300 import _binding as B  # noqa: E402

M32 = 0xFFFFFFFF


def _start(n_threads):
    g = np.arange(n_threads, dtype=np.uint64)[:, None]
    return 8 * g + np.arange(8, dtype=np.uint64)[None, :] + 1  # [thread][chain]


def _expected_int(op, n_threads, iters):
    x = _start(n_threads)
    for _ in range(iters):
        if op == B.SPIN_PIPE_MUL_WIDE:
            lo = x & M32
            x = (lo * np.uint64(0xD2511F53) + x) & np.uint64(0xFFFFFFFFFFFFFFFF)
        elif op == B.SPIN_PIPE_MAD_HI:
            x = (((x * np.uint64(0xCD9E8D57)) >> np.uint64(32)) + np.uint64(0x9E3779B9)) & np.uint64(M32)
        elif op == B.SPIN_PIPE_LOP3:
            x = x ^ np.roll(x, -1, axis=1) ^ np.roll(x, -2, axis=1)
        else:
            x = (x + np.roll(x, -1, axis=1) + np.roll(x, -2, axis=1)) & np.uint64(M32)
    if op == B.SPIN_PIPE_MUL_WIDE:
        x = (x & np.uint64(M32)) ^ (x >> np.uint64(32))
    return np.bitwise_xor.reduce(x, axis=1).astype(np.uint32)


def _run(op, bpsm, iters):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    clocks = torch.zeros(3 * sms * bpsm, dtype=torch.int64, device="cuda")
    sink = torch.zeros(sms * bpsm * 256, dtype=torch.int32, device="cuda")
    n = B.spin_pipe_probe(op, bpsm, iters, clocks, sink, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert n == sms
    c = clocks.view(-1, 3).cpu().numpy()
    # every CTA recorded an increasing clock pair and a valid SM index
    assert (c[:, 1] >= c[:, 0]).all() and (c[:, 0] > 0).all() and (c[:, 2] >= 0).all() and (c[:, 2] < sms).all()
    return c, sink.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("op", [B.SPIN_PIPE_MUL_WIDE, B.SPIN_PIPE_MAD_HI, B.SPIN_PIPE_LOP3, B.SPIN_PIPE_IADD3])
def test_integer_chains_match_host_emulation(op):
    iters = 5
    c, sink = _run(op, 2, iters)
    assert (c[:, 1] > c[:, 0]).all()
    assert np.array_equal(sink, _expected_int(op, sink.size, iters))


def _float_start(n_threads):
    g = np.arange(n_threads, dtype=np.float64)[:, None]
    return (1.0 + (8 * g + np.arange(8)[None, :]) * 2.0 ** -20).astype(np.float32)


def _sum32(f32):
    acc = np.zeros(f32.shape[0], np.float32)
    for c in range(8):
        acc = (acc + f32[:, c]).astype(np.float32)
    return acc


@pytest.mark.parametrize("op", [B.SPIN_PIPE_FFMA, B.SPIN_PIPE_MUFU_RSQ])
def test_float_chains_match_host_emulation(op):
    """Zero iterations return the sum of the start values bit for bit; after a
    few iterations the sums agree with an FP64 emulation of the chains (FFMA
    to FP32 rounding, the approximate reciprocal square root to its stated
    relative error, which the map x -> x^(-1/2) does not amplify)."""
    _, sink0 = _run(op, 1, 0)
    start = _float_start(sink0.size)
    assert np.array_equal(sink0.view(np.float32), _sum32(start))
    iters = 6
    c, sink = _run(op, 1, iters)
    assert (c[:, 1] > c[:, 0]).all()
    f = start.astype(np.float64)
    for _ in range(iters):
        f = f * float(np.float32(0.999)) + float(np.float32(0.001)) if op == B.SPIN_PIPE_FFMA else 1.0 / np.sqrt(f)
    want = f.sum(axis=1)
    got = sink.view(np.float32).astype(np.float64)
    assert np.max(np.abs(got - want) / want) < 4e-6


def test_invalid_arguments_are_rejected():
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    clocks = torch.zeros(3 * sms * 9, dtype=torch.int64, device="cuda")
    sink = torch.zeros(sms * 9 * 256, dtype=torch.int32, device="cuda")
    for op, bpsm in ((6, 1), (-1, 1), (B.SPIN_PIPE_LOP3, 0), (B.SPIN_PIPE_LOP3, 9)):
        with pytest.raises(B.SpinError):
            B.spin_pipe_probe(op, bpsm, 1, clocks, sink)
