"""Tensor-core X-engine (tcgen05 Gram matrices) against the exact oracle Gram.

Inputs are seeded codes drawn on the host (never produced by the CUDA path):
int8 codes carried as BF16, int8 codes as bytes (widened to BF16 on chip by
the kernel the int8 pipeline uses) and e4m3 bytes.  With int8 codes every product is
exact and FP32 sums are exact while partial sums stay below 2^24, which
holds for K <= 1024 (1024 * 127^2 < 2^24): there the result must be
bit-exact.  Longer sums and e4m3 are checked against the FP32 accumulation
bound |G - G_exact| <= K * 2^-24 * sum_k |q_r q_s|.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import requant_oracle as rq  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_20640_gb300.build import build_library
    build_library()


def _corr():
    from paper_2604_20640_gb300 import Correlator
    return Correlator(4, 1, 64, 4, 16)


def _bf16_bits(v):
    return (np.asarray(v, np.float32).view(np.uint32) >> 16).astype(np.uint16)


def _run_gram(c, Qbytes, n_chan, k_pitch, K, dtype):
    Qd = torch.from_numpy(Qbytes).to(DEV)
    G = torch.full((n_chan, 128, 128), float("nan"), dtype=torch.float32, device=DEV)
    c.gram_dev(Qd, n_chan, k_pitch, K, dtype, G)
    torch.cuda.synchronize()
    assert c.device_status() == 0
    return G.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("rows,K,k_pitch", [(128, 1024, 2048), (16, 1000, 2048), (100, 256, 512), (128, 64, 256)])
def test_int8_gram_bit_exact(rows, K, k_pitch):
    from paper_2604_20640_gb300 import CORR_INT8
    rng = np.random.default_rng(rows + K)
    n_chan = 6
    codes = np.zeros((n_chan, 128, k_pitch // 2), np.int64)
    codes[:, :rows, :K] = rng.integers(-127, 128, size=(n_chan, rows, K))
    codes[:, :rows, K:] = rng.integers(-127, 128, size=(n_chan, rows, k_pitch // 2 - K))  # beyond K: ignored
    Q = _bf16_bits(codes).view(np.uint8).reshape(n_chan, 128, k_pitch)
    G = _run_gram(_corr(), Q, n_chan, k_pitch, K, CORR_INT8)
    ref = rq.gram(codes[:, :, :K])
    np.testing.assert_array_equal(G, ref.astype(np.float64))


def test_int8_gram_long_sums_within_fp32_bound():
    from paper_2604_20640_gb300 import CORR_INT8
    rng = np.random.default_rng(7)
    n_chan, K = 4, 4096
    codes = rng.integers(-127, 128, size=(n_chan, 128, K))
    codes[:, :, ::3] = 127                               # large positive sums
    Q = _bf16_bits(codes).view(np.uint8).reshape(n_chan, 128, 2 * K)
    G = _run_gram(_corr(), Q, n_chan, 2 * K, K, CORR_INT8)
    ref = rq.gram(codes).astype(np.float64)
    bound = K * 2.0 ** -24 * rq.gram(np.abs(codes)).astype(np.float64)
    assert np.all(np.abs(G - ref) <= bound + 1e-9)


def test_e4m3_gram_within_fp32_bound():
    from paper_2604_20640_gb300 import CORR_FP8
    rng = np.random.default_rng(9)
    n_chan, K = 5, 2048
    vals = rq.e4m3_round(rng.standard_normal((n_chan, 128, K)) * 40.0)
    # encode grid values as bytes through the decode table
    table = rq.e4m3_decode(np.arange(256, dtype=np.uint8))
    lut = {float(v): i for i, v in enumerate(table) if not np.isnan(v)}
    lut[0.0] = 0
    Qb = np.vectorize(lambda v: lut[float(v)])(vals).astype(np.uint8)
    G = _run_gram(_corr(), Qb, n_chan, K, K, CORR_FP8)
    dec = rq.e4m3_decode(Qb)
    ref = rq.gram(dec)
    bound = K * 2.0 ** -24 * rq.gram(np.abs(dec))
    assert np.all(np.abs(G - ref) <= bound + 1e-9)


def test_gram_rejects_bad_layout():
    from paper_2604_20640_gb300 import CorrError, CORR_INT8
    c = _corr()
    Q = torch.zeros((2, 128, 200), dtype=torch.uint8, device=DEV)
    G = torch.zeros((2, 128, 128), dtype=torch.float32, device=DEV)
    with pytest.raises(CorrError):
        c.gram_dev(Q, 2, 200, 64, CORR_INT8, G)


@pytest.mark.parametrize("rows,K,k_pitch", [(128, 1024, 1024), (16, 1000, 1024), (100, 130, 256), (128, 64, 128)])
def test_int8_byte_gram_bit_exact(rows, K, k_pitch):
    """int8 codes stored as bytes: the kernel widens each 128-code tile to
    two swizzled BF16 operand tiles; exact products, exact FP32 sums up to
    K = 1024 -> bit-exact; codes beyond K (in the row pitch) are ignored."""
    from paper_2604_20640_gb300 import CORR_INT8_BYTES
    rng = np.random.default_rng(rows + 7 * K)
    n_chan = 5
    codes = np.zeros((n_chan, 128, k_pitch), np.int64)
    codes[:, :rows, :K] = rng.integers(-127, 128, size=(n_chan, rows, K))
    codes[:, :rows, K:] = rng.integers(-127, 128, size=(n_chan, rows, k_pitch - K))
    Q = codes.astype(np.int8).view(np.uint8)
    G = _run_gram(_corr(), Q, n_chan, k_pitch, K, CORR_INT8_BYTES)
    np.testing.assert_array_equal(G, rq.gram(codes[:, :, :K]).astype(np.float64))


def test_int8_byte_gram_long_sums_within_fp32_bound():
    from paper_2604_20640_gb300 import CORR_INT8_BYTES
    rng = np.random.default_rng(3)
    n_chan, K, k_pitch = 3, 4096, 4096
    codes = rng.integers(-127, 128, size=(n_chan, 128, K)).astype(np.int64)
    G = _run_gram(_corr(), codes.astype(np.int8).view(np.uint8), n_chan, k_pitch, K, CORR_INT8_BYTES)
    ref = rq.gram(codes).astype(np.float64)
    bound = K * 2.0 ** -24 * np.einsum('crk,csk->crs', np.abs(codes).astype(np.float64), np.abs(codes).astype(np.float64))
    assert np.all(np.abs(G - ref) <= bound)


def _words(q_re, q_im):
    """Code words [K][n_pairs][n_chan] uint32 from codes q_re, q_im [N][K][n_chan]:
    bytes Re V_2p, Im V_2p, Re V_2p+1, Im V_2p+1 (low byte first); the bytes
    of inputs past N are zero."""
    N, K, n_chan = q_re.shape
    n_pairs = (N + 3) // 4 * 2          # n_in padded to a multiple of 4, in pairs
    b = np.zeros((K, n_pairs, n_chan, 4), np.int64)
    for a in range(N):
        b[:, a // 2, :, 2 * (a % 2)] = q_re[a]
        b[:, a // 2, :, 2 * (a % 2) + 1] = q_im[a]
    u = (b & 0xFF).astype(np.uint32)
    return u[..., 0] | (u[..., 1] << 8) | (u[..., 2] << 16) | (u[..., 3] << 24)


@pytest.mark.parametrize("n_in,n_chan,K", [(64, 8, 1024), (20, 12, 100), (7, 4, 64), (64, 1024, 320), (33, 16, 1)])
def test_int8_word_gram_bit_exact(n_in, n_chan, K):
    """The int8 pipeline's form: the Gram kernel reads the F-engine's code
    words [K][pair][channel] directly (four channels a CTA, raw boxes of 64
    spectra by 3D TMA, widened to BF16 in rows Re a = a, Im a = N + a);
    exact products and FP32 sums up to K = 1024 -> bit-exact on the 2N x 2N
    block the visibilities use (ragged K, odd N, one spectrum)."""
    from paper_2604_20640_gb300 import Correlator, CORR_INT8_WORDS
    rng = np.random.default_rng(n_in * 1000 + n_chan + K)
    q_re = rng.integers(-127, 128, size=(n_in, K, n_chan)).astype(np.int64)
    q_im = rng.integers(-127, 128, size=(n_in, K, n_chan)).astype(np.int64)
    W = _words(q_re, q_im)
    c = Correlator(n_in, 1, 64, 4, 16)
    G = _run_gram(c, W.view(np.uint8).reshape(-1), n_chan, 0, K, CORR_INT8_WORDS)
    c.close()
    ref = rq.gram(rq.stacked_rows(q_re, q_im))
    n2 = 2 * n_in
    np.testing.assert_array_equal(G[:, :n2, :n2], ref[:, :n2, :n2].astype(np.float64))


@pytest.mark.parametrize("n_in,n_chan,K", [(64, 8, 1024), (20, 12, 100), (7, 4, 64), (64, 1024, 320), (33, 16, 1)])
def test_e4m3_word_gram(n_in, n_chan, K):
    """The e4m3 pipeline's form: the same code words holding e4m3 bytes, 128
    spectra an operand tile (two raw boxes; a box wholly past K is zeros).
    Against the exact Gram of the decoded codes within the FP32 summation
    bound, and bit for bit against the row-major e4m3 Gram of the same codes
    (same spectra in the same order through the same MMA steps) on the
    2N x 2N block the visibilities use."""
    from paper_2604_20640_gb300 import Correlator, CORR_FP8, CORR_FP8_WORDS
    rng = np.random.default_rng(n_in * 1000 + n_chan + K + 5)
    finite = np.array([b for b in range(256) if (b & 0x7F) != 0x7F], np.int64)   # no NaN codes
    q_re = rng.choice(finite, size=(n_in, K, n_chan))
    q_im = rng.choice(finite, size=(n_in, K, n_chan))
    W = _words(q_re, q_im)
    c = Correlator(n_in, 1, 64, 4, 16)
    G = _run_gram(c, W.view(np.uint8).reshape(-1), n_chan, 0, K, CORR_FP8_WORDS)
    k_pitch = (K + 127) // 128 * 128
    Qb = np.zeros((n_chan, 128, k_pitch), np.uint8)
    Qb[:, :n_in, :K] = q_re.transpose(2, 0, 1)
    Qb[:, n_in:2 * n_in, :K] = q_im.transpose(2, 0, 1)
    G_rm = _run_gram(c, Qb, n_chan, k_pitch, K, CORR_FP8)
    c.close()
    n2 = 2 * n_in
    dec = rq.e4m3_decode(Qb[:, :n2, :K])
    ref = rq.gram(dec)
    bound = K * 2.0 ** -24 * rq.gram(np.abs(dec))
    assert np.all(np.abs(G[:, :n2, :n2] - ref) <= bound + 1e-30)
    np.testing.assert_array_equal(G[:, :n2, :n2], G_rm[:, :n2, :n2])


def test_int8_word_gram_rejects_bad_layout():
    from paper_2604_20640_gb300 import Correlator, CorrError, CORR_EINVAL, CORR_INT8_WORDS
    c = Correlator(8, 1, 64, 4, 16)
    W = torch.zeros(64 * 4 * 6, dtype=torch.uint32 if hasattr(torch, "uint32") else torch.int32, device=DEV)
    G = torch.empty((6, 128, 128), device=DEV)
    with pytest.raises(CorrError) as e:
        c.gram_dev(W, 6, 0, 64, CORR_INT8_WORDS, G)             # n_chan not a multiple of 4
    assert e.value.code == CORR_EINVAL
    c.close()
