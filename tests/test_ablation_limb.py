"""Tensor-core limb ablations of the mod-p GEMM (tn_modp_gemm_limb on integer
MMAs, tn_modp_gemm_umma on tcgen05): exact against plain integer arithmetic
on a small case, and bit-identical to the CUDA-core path (tn_contract_pair
on the same buffers) on larger ones, including k longer than one exact
8192-term diagonal block."""
import os

import numpy as np
import pytest

from paper_2501_00227_gb300 import tn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_00227_gb300 import build as B
    B.build()


def _residues(rng, primes, shape):
    out = np.empty((len(primes),) + shape, dtype=np.uint32)
    for q, p in enumerate(primes):
        out[q] = rng.integers(0, p, size=shape, dtype=np.int64).astype(np.uint32)
    return out


def _limb(primes, A, B, batch, m, n, k, fn=None):
    fn = fn or tn.tn_modp_gemm_limb
    a, b = torch.from_numpy(A.view(np.int32)).cuda(), torch.from_numpy(B.view(np.int32)).cuda()
    c = torch.zeros(len(primes) * batch * m * n, dtype=torch.int32, device="cuda")
    fn(primes, a.data_ptr(), b.data_ptr(), c.data_ptr(), batch, m, n, k, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return c.cpu().numpy().view(np.uint32).reshape(len(primes), batch, m, n)


def test_limb_gemm_exact_small():
    primes = tn.PRIMES31[:2]
    rng = np.random.default_rng(3)
    batch, m, n, k = 1, 64, 32, 64
    A = _residues(rng, primes, (batch, m, k))
    B = _residues(rng, primes, (batch, n, k))
    got = _limb(primes, A, B, batch, m, n, k)
    for q, p in enumerate(primes):
        ref = (A[q, 0].astype(object) @ B[q, 0].astype(object).T) % p
        assert (got[q, 0].astype(object) == ref).all()


@pytest.mark.parametrize("batch,m,n,k,nprimes", [(2, 128, 64, 256, 3), (1, 64, 32, 16384, 1), (4, 64, 64, 32, 4)])
def test_limb_gemm_matches_cuda_core_path(batch, m, n, k, nprimes):
    primes = tn.PRIMES31[:nprimes]
    rng = np.random.default_rng(batch * 1000 + k)
    A = _residues(rng, primes, (batch, m, k))
    B = _residues(rng, primes, (batch, n, k))
    got = _limb(primes, A, B, batch, m, n, k)
    # the same contraction as a pairwise step: labels k | m | b for A, k | n | b for B, output n | m | b
    lk, lm, ln, lb = (list(range(s, s + w)) for s, w in
                      ((0, int(np.log2(k))), (40, int(np.log2(m))), (60, int(np.log2(n))), (80, int(np.log2(batch)))))
    a = torch.from_numpy(A.view(np.int32).reshape(-1)).cuda()
    b = torch.from_numpy(B.view(np.int32).reshape(-1)).cuda()
    c = torch.zeros(nprimes * batch * m * n, dtype=torch.int32, device="cuda")
    tn.tn_contract_pair("modp", primes, a.data_ptr(), lk + lm + lb, b.data_ptr(), lk + ln + lb, ln + lm + lb,
                        c.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    ref = c.cpu().numpy().view(np.uint32).reshape(nprimes, batch, m, n)
    assert (got == ref).all()


def test_limb_gemm_rejects_unsupported_shapes():
    with pytest.raises(tn.TNError) as ei:
        tn.tn_modp_gemm_limb(tn.PRIMES31[:1], 1, 1, 1, 1, 48, 32, 32, 0)
    assert ei.value.code == tn.TN_EINVAL


def test_umma_gemm_exact_small():
    primes = tn.PRIMES31[:1]
    rng = np.random.default_rng(11)
    batch, m, n, k = 1, 128, 64, 64
    A = _residues(rng, primes, (batch, m, k))
    B = _residues(rng, primes, (batch, n, k))
    got = _limb(primes, A, B, batch, m, n, k, tn.tn_modp_gemm_umma)
    ref = (A[0, 0].astype(object) @ B[0, 0].astype(object).T) % primes[0]
    assert (got[0, 0].astype(object) == ref).all()


@pytest.mark.parametrize("batch,m,n,k,nprimes", [(2, 256, 128, 256, 3), (1, 128, 64, 1024, 4)])
def test_umma_gemm_matches_integer_mma(batch, m, n, k, nprimes):
    primes = tn.PRIMES31[:nprimes]
    rng = np.random.default_rng(batch * 77 + k)
    A = _residues(rng, primes, (batch, m, k))
    B = _residues(rng, primes, (batch, n, k))
    assert (_limb(primes, A, B, batch, m, n, k, tn.tn_modp_gemm_umma) == _limb(primes, A, B, batch, m, n, k)).all()


def _umma_steps(plan, nprimes):
    """GEMM-shaped mod-p steps the tensor-core route takes (M % 128, N % 64,
    K % 64 == 0; the operands of such steps are intermediates)."""
    si = tn.tn_plan_step_info(plan.handle, "modp", nprimes)
    return int(((si[:, 7] >= 7) & (si[:, 8] >= 6) & (si[:, 9] >= 6)).sum())


@pytest.mark.parametrize("spec,nprimes", [("reg3:140:2", 3), ("ksg:20:0.8:1", 4)])
def test_contraction_through_tensor_core_route(spec, nprimes, monkeypatch):
    """A whole contraction with its GEMM-shaped mod-p steps on the tcgen05
    limb GEMM (one launch per step, TN_UMMA=1) gives the residues of the
    executor and of the oracle (Sec. 5.1)."""
    import graphgen as g
    import oracle as O
    n, e = g.by_name(spec)
    primes = tn.PRIMES31[:nprimes]
    p = tn.Plan(n, e, nrepeat=10, seed=1)
    try:
        assert _umma_steps(p, nprimes) >= 2
        ref = p.contract("modp", primes)["residues"]
        monkeypatch.setenv("TN_EXEC", "0")
        monkeypatch.setenv("TN_UMMA", "1")
        got = p.contract("modp", primes)["residues"]
        monkeypatch.setenv("TN_UMMA", "0")
        plain = p.contract("modp", primes)["residues"]
        assert got == plain == ref
        if spec.startswith("reg3"):
            O.set_threads(os.cpu_count() or 1)
            assert got == O.count_modp(n, e, p.order, primes)
    finally:
        p.close()
