"""The Gram matrices of the weight factorisations (dh2_gram), on the GPU.

The Cholesky QR of the stacked weights (Section 3.2, the QR of the stacked coupling and
father-weight rows) starts from G = Z^* Z.  For FP32 stacks of more than 32 columns the
library forms G from exact integer digit products on the tensor cores (dh2_options.gram_tc);
these tests pin that product against numpy, which is exact or FP64-accurate here:

- integer data (16-bit integers times a power of two per column): every digit product, every
  FP32 accumulator sum and every FP64 partial sum is exact, so G must equal the exact integer
  Gram bit for bit -- an accumulation that rounded anywhere would miss it;
- general FP32 data with row scales over six decades: the error stays within the stated bound
  of about 2^-43 max|z_m| max|z_n| per row;
- the FP64 CUDA-core Gram (gram_tc = 0) on the same data, and a build with either Gram.
"""
import numpy as np
import pytest


pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_04384_gb300.build import build

    build()


def _integer_matrix(rows, cols, ld, seed):
    """16-bit signed integers (real and imaginary parts) times 2^k_j per column j."""
    g = np.random.default_rng(seed)
    re = g.integers(-(2 ** 15) + 1, 2 ** 15, size=(rows, ld))
    im = g.integers(-(2 ** 15) + 1, 2 ** 15, size=(rows, ld))
    k = g.integers(-20, 21, size=ld)
    # a few sparse columns and one zero column: exponents and digits of small maxima
    re[:, 1] = np.where(g.random(rows) < 0.05, re[:, 1], 0)
    im[:, 1] = 0
    if ld > 3:
        re[:, 3] = 0
        im[:, 3] = 0
    return re, im, k


def _exact_gram(re, im, k, cols):
    """Z^* Z of Z = (re + i im) 2^k from int64 sums (exact) scaled by 2^(k_m + k_n)."""
    a, b = re[:, :cols].astype(np.int64), im[:, :cols].astype(np.int64)
    gre = a.T @ a + b.T @ b
    gim = a.T @ b - b.T @ a
    assert np.abs(gre).max() < 2 ** 53 and np.abs(gim).max() < 2 ** 53
    sc = np.ldexp(1.0, (k[:cols, None] + k[None, :cols]).astype(np.int64))
    return gre.astype(np.float64) * sc + 1j * (gim.astype(np.float64) * sc)


@pytest.mark.parametrize("rows,cols,ld", [(5000, 125, 125), (2100, 216, 216), (777, 40, 48), (4099, 64, 64),
                                          (3000, 32, 32), (300, 100, 128), (2500, 17, 24), (6000, 5, 5)])
@pytest.mark.parametrize("gram_tc", [1, 0])
def test_gram_exact_on_integer_data(rows, cols, ld, gram_tc):
    import torch

    import paper_1809_04384_gb300 as dh2

    re, im, k = _integer_matrix(rows, cols, ld, seed=rows + cols)
    z = (np.ldexp(re.astype(np.float64), k) + 1j * np.ldexp(im.astype(np.float64), k)).astype(np.complex64)
    assert np.array_equal(z.real.astype(np.float64), np.ldexp(re.astype(np.float64), k))   # exact in FP32
    zt = torch.from_numpy(z).cuda()[:, :cols]   # row pitch ld
    g = dh2.dh2_gram(zt, gram_tc=gram_tc).cpu().numpy()
    want = _exact_gram(re, im, k, cols)
    assert np.array_equal(g.real, want.real) and np.array_equal(g.imag, want.imag)


def _float_matrix(rows, cols, seed):
    g = np.random.default_rng(seed)
    z = g.standard_normal((rows, cols)) + 1j * g.standard_normal((rows, cols))
    z *= 10.0 ** g.uniform(-3, 3, size=(rows, 1))      # weighted stack rows
    z[:, 0] *= 1e-6                                     # one column far below the others
    return z.astype(np.complex64)


@pytest.mark.parametrize("rows,cols", [(3000, 125), (1500, 216), (5000, 64), (600, 33), (4000, 32), (2000, 9)])
def test_gram_tc_error_bound_on_float_data(rows, cols):
    import torch

    import paper_1809_04384_gb300 as dh2

    z = _float_matrix(rows, cols, seed=7 * rows + cols)
    z64 = z.astype(np.complex128)
    ref = z64.conj().T @ z64                              # FP64: error ~ 1e-16 relative
    zt = torch.from_numpy(z).cuda()
    g = dh2.dh2_gram(zt, gram_tc=1).cpu().numpy()
    mx = np.maximum(np.abs(z64.real), np.abs(z64.imag)).max(axis=0)
    bound = 2.0 ** -42 * rows * np.outer(mx, mx) * 2      # two real products per complex entry
    assert np.all(np.abs(g - ref) <= bound + 1e-14 * np.abs(ref))
    assert np.linalg.norm(g - ref) <= 1e-12 * np.linalg.norm(ref)
    # the Hermitian structure is exact (one triangle mirrored), the diagonal real
    assert np.array_equal(g, g.conj().T)
    # the FP64 CUDA-core Gram on the same data
    g0 = dh2.dh2_gram(zt, gram_tc=0).cpu().numpy()
    assert np.linalg.norm(g0 - ref) <= 1e-14 * np.linalg.norm(ref)


def test_gram_rejects_non_finite_input():
    import torch

    import paper_1809_04384_gb300 as dh2

    z = _float_matrix(200, 80, seed=3)
    z[17, 5] = np.nan
    for gram_tc in (1, 0):
        with pytest.raises(dh2.DH2Error) as e:
            dh2.dh2_gram(torch.from_numpy(z).cuda(), gram_tc=gram_tc)
        assert e.value.status == dh2.DH2_ENUMERIC


@pytest.mark.parametrize("name", ["dir320m6", "dir1280", "dir320m5"])
def test_build_with_either_gram(name):
    """The mixed form with the tensor-core Gram (default) and with the FP64 CUDA-core Gram:
    the same ranks (up to ties at the threshold) and products that agree to FP32 rounding
    of the stored data."""
    import torch

    import paper_1809_04384_gb300 as dh2
    from tests.cases import mesh, params
    from tests.gpu_common import rel, x_vector

    v, f = mesh(name)
    p = params(name)
    tree = dh2.Tree(v, f, leaf_max=p["leaf"])
    mats = [dh2.Matrix(tree, p["kappa"], p["m"], p["eta2"], p["eps"], eta1=p["eta1"], gram_tc=t) for t in (1, 0)]
    info = mats[0].get_info()
    # K_TSQR (wide stacks) and K_TSQR_NARROW (at most 32 columns) on the tensor cores or in FP64
    assert info.kernel_work_kind[5] == 4 and mats[1].get_info().kernel_work_kind[5] == 2
    assert info.kernel_work_kind[13] == 4 and mats[1].get_info().kernel_work_kind[13] == 2
    # where stacks taller than wide occurred, their Gram ran on the tensor cores
    assert (info.kernel_launches[5] > 0) == (info.kernel_work[5] > 0)
    assert (info.kernel_launches[13] > 0) == (info.kernel_work[13] > 0)
    (r1, c1), (r0, c0) = mats[0].ranks(), mats[1].ranks()
    assert np.mean(r1 != r0) <= 0.01 and np.mean(c1 != c0) <= 0.01
    x = torch.from_numpy(x_vector(tree.n)).to(torch.complex64).cuda()
    y1, y0 = (m.matvec(x).cpu().numpy().astype(np.complex128) for m in mats)
    assert rel(y1, y0) <= (1e-5 if np.array_equal(r1, r0) and np.array_equal(c1, c0) else 2 * p["eps"])
