"""GPU parity of the split-BF16 tensor-core contraction (kite_inner_products) against
the plain FP64 definition C = scale * conj(A) B^T (the contraction of Eq. Gammanm).

Error model of the GPU path: each FP32 input is represented as hi + lo (bf16 each) to
relative 2^-17, the dropped lo*lo term is 2^-16 relative per product, FP32 sums inside
sub-chunks of `sub_k` products, FP32 again over `fold` sub-chunks (registers) and FP64
above.  The bar, written per test, is a bound on
|C_gpu - C_ref| relative to sum_i |A_n(i)| |B_m(i)| (the scale of the terms)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

kite = pytest.importorskip("paper_1910_05194_gb300")


@pytest.fixture(scope="module")
def ctx():
    c = kite.Context(0)
    yield c
    c.close()


def run(ctx, A, B, scale=1.0, sub_k=0, products=0, fold=0):
    M, N = A.shape
    M2 = B.shape[0]
    A32 = np.ascontiguousarray(A.astype(np.complex64))
    B32 = np.ascontiguousarray(B.astype(np.complex64))
    C = np.zeros((M, M2), np.complex128)
    kite.inner_products(ctx, A32, B32, M, M2, N, scale, C, sub_k, products, fold)
    ref = oracle.inner_products(A32, B32, scale)
    bound = np.abs(scale) * (np.abs(A32).astype(np.float64) @ np.abs(B32).astype(np.float64).T)
    return C, ref, bound


@pytest.mark.parametrize("M,M2,N", [(1, 1, 1), (128, 128, 4096), (200, 77, 3001),
                                    (257, 300, 12345), (64, 512, 65536)])
def test_random_families(ctx, M, M2, N):
    A = synth.gaussian_vectors(N, M, seed=M * 7 + N)
    B = synth.gaussian_vectors(N, M2, seed=M2 * 11 + N)
    C, ref, bound = run(ctx, A, B, scale=1.0 / N)
    assert np.all(np.abs(C - ref) <= 2.0**-13 * bound + 1e-300)


def test_aligned_terms_long_k_accumulation(ctx):
    """All-positive terms (the diagonal mu_00 = <h r|h r> is of this kind).  Two error
    sources are separated: bf16-representable inputs (lo = 0) isolate the FP32 accumulation
    inside a sub-chunk; general inputs add the split error, which with three products has a
    one-signed lo*lo bias of up to ~5e-6 and with four products is unbiased."""
    N = 1 << 20
    g = np.random.Generator(np.random.PCG64(3))
    a = (0.5 + g.random(N)).astype(np.float32)
    exact_bf16 = (a.view(np.uint32) & np.uint32(0xFFFF0000)).view(np.float32)
    res = {}
    for name, vec in (("bf16-exact", exact_bf16), ("general", a)):
        A = vec[None, :].astype(np.complex64)
        for products in (3, 4):
            for sub_k in (256, 512, 1024, 4096):
                # fold = 1: every sub-chunk straight to FP64, the sub-chunk alone measured
                C, ref, bound = run(ctx, A, A, scale=1.0 / N, sub_k=sub_k, products=products, fold=1)
                res[(name, products, sub_k)] = abs(C[0, 0] - ref[0, 0]) / abs(ref[0, 0])
        for fold in (4, 16, 64):
            C, ref, bound = run(ctx, A, A, scale=1.0 / N, sub_k=512, products=4, fold=fold)
            res[(name, 4, 512, "fold", fold)] = abs(C[0, 0] - ref[0, 0]) / abs(ref[0, 0])
    for k, v in sorted(res.items(), key=str):
        print(f"{k}: relative error {v:.3e}")
    # default path (4 products, 512-product sub-chunks, 16 of them summed in FP32) well
    # inside the 1e-5 bar; the FP32 accumulation error grows linearly with the sub-chunk
    # length, while the second FP32 level adds ~fold/4 * 2^-24 at most
    assert res[("general", 4, 512)] <= 4e-6
    assert res[("general", 4, 512, "fold", 16)] <= res[("general", 4, 512)] + 5e-7
    assert res[("bf16-exact", 4, 256)] <= 1e-12  # bf16 products sum exactly over 256 terms
    assert res[("general", 4, 256)] < res[("general", 4, 4096)]


def test_host_and_device_buffers(ctx):
    torch = pytest.importorskip("torch")
    M, M2, N = 96, 130, 5000
    A = synth.gaussian_vectors(N, M, seed=1).astype(np.complex64)
    B = synth.gaussian_vectors(N, M2, seed=2).astype(np.complex64)
    Ad = torch.from_numpy(A.view(np.float32)).cuda()
    Bd = torch.from_numpy(B.view(np.float32)).cuda()
    Cd = torch.zeros((M, M2, 2), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()  # inputs produced on torch's stream must be complete
    kite.inner_products(ctx, Ad, Bd, M, M2, N, 1.0, Cd)
    C = Cd.cpu().numpy()
    C = C[..., 0] + 1j * C[..., 1]
    ref = oracle.inner_products(A, B)
    bound = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    Ch = np.zeros((M, M2), np.complex128)
    kite.inner_products(ctx, A, B, M, M2, N, 1.0, Ch)  # host buffers, same inputs
    ratio = np.abs(C - ref) / (2.0**-13 * bound)
    worst = np.unravel_index(np.argmax(ratio), ratio.shape)
    assert np.max(ratio) <= 1.0, (worst, C[worst], Ch[worst], ref[worst])
    assert np.max(np.abs(C - Ch)) <= 1e-12 * np.max(np.abs(ref))
