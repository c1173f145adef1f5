"""GPU parity of the step's small kernels through the C ABI: the residual
stand-in network F(u) = u + theta, the Adam update of Algorithm 2 (Sec.
4.1.3) against the FP64 oracle over several steps (vectorised and scalar
paths, one or two gradient sets, BF16 gradients), and the per-iteration
draws loaded on the device from a resident table (Algorithm 2 draws a
sketch and G rotations every iteration), eagerly and from a CUDA graph."""
import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2411_05771_gb300 import skei
    return skei


def dev(a, dtype=torch.float32):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


@pytest.mark.parametrize("count,n", [(1, 4096), (3, 1000), (2, 37), (5, 1)])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_residual_add(S, count, n, dtype):
    rng = np.random.default_rng(count * n)
    u = dev(rng.standard_normal((count, n)), dtype)
    theta = dev(rng.standard_normal(n))
    out = S.residual_add(u, theta)
    # one FP32 addition, correctly rounded (the FP64 sum of these operands is
    # exact), then the storage type's rounding
    ref = dev(host(u) + host(theta)[None]).to(dtype)
    assert torch.equal(out, ref)


# n % 4 == 0 takes the 16-byte path, the others the scalar one
@pytest.mark.parametrize("n,c1,c2,gdt", [(4096, 1, 0, torch.float32), (4096, 1, 4, torch.float32),
                                         (1001, 2, 1, torch.float32), (512, 1, 4, torch.bfloat16)])
def test_adam_matches_oracle_over_steps(S, n, c1, c2, gdt):
    rng = np.random.default_rng(n + c1 + c2)
    theta = dev(rng.standard_normal(n))
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    t_o, m_o, v_o = host(theta), np.zeros(n), np.zeros(n)
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    for k in range(1, 8):
        g1 = dev(rng.standard_normal((c1, n)), gdt)
        g2 = dev(rng.standard_normal((c2, n)), gdt) if c2 else None
        step.fill_(k)
        S.adam_step(theta, m, v, step[0], g1, g2, lr=5e-4)
        g = host(g1).sum(axis=0) + (host(g2).sum(axis=0) if c2 else 0.0)
        t_o, m_o, v_o = O.adam_step(t_o, g, m_o, v_o, k)
    # FP32 state: the moments to a few FP32 roundings; theta to the half-ulp
    # roundings of its 7 FP32 updates plus 1e-8 (each update is ~lr = 5e-4:
    # a 1e-4 relative error in it would show)
    # (m's terms are ~0.1 and may cancel: an absolute floor of 1e-7)
    np.testing.assert_allclose(host(m), m_o, rtol=2e-6, atol=1e-7)
    np.testing.assert_allclose(host(v), v_o, rtol=2e-6, atol=1e-10)
    ulp = np.spacing(np.abs(t_o).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(host(theta) - t_o) <= 7 * ulp + 1e-8)


@pytest.mark.parametrize("row_bytes", [1744, 37])
def test_step_draws_walks_the_table_and_stops_at_its_end(S, row_bytes):
    rng = np.random.default_rng(row_bytes)
    rows = 5
    table = torch.tensor(rng.integers(0, 256, (rows, row_bytes), dtype=np.uint8), device="cuda")
    out = torch.zeros(row_bytes, dtype=torch.uint8, device="cuda")
    counter = torch.zeros(1, dtype=torch.int32, device="cuda")
    for r in range(rows):
        S.step_draws(table, counter, out)
        assert torch.equal(out, table[r])
        assert counter.item() == r + 1
    # past the end: nothing copied, the counter becomes -1 and stays there
    S.step_draws(table, counter, out)
    assert counter.item() == -1 and torch.equal(out, table[rows - 1])
    S.step_draws(table, counter, out)
    assert counter.item() == -1
    with pytest.raises(ValueError):
        S.step_draws(table, counter, out[:-1])


def test_step_draws_in_a_graph_give_each_replay_its_row(S):
    """A captured [draws, consumer] pair replayed K times: replay k sees row
    k (here the consumer adds the row's floats to an accumulator)."""
    K, n = 6, 64
    table = dev(np.arange(K * n, dtype=np.float64).reshape(K, n))
    row = torch.zeros(n, device="cuda")
    acc = torch.zeros(n, device="cuda")
    counter = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=st):
            S.step_draws(table, counter, row)
            acc.add_(row)
        counter.zero_()
        acc.zero_()
        for _ in range(K):
            graph.replay()
    st.synchronize()
    assert counter.item() == K
    assert torch.equal(acc, table.sum(dim=0))
