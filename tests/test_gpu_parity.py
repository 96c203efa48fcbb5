"""Parity of the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (|K_gpu - K_oracle|, elementwise):
  FP64        1e-10  (the FP64 parity bar)
  FP32_SPLIT  1e-6   (the low-precision bar; measured ~1e-8 at n = 784)
  FP32        2e-5 for n <= 64 and 1e-4 at n = 784 (plain FP32 is the fast path
              without compensation: its coherent rounding error grows with n)
log K is compared where the oracle's K exceeds 1e-300.
"""
import numpy as np
import pytest

from paper_2405_02630_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32_split": 1e-6, "fp32": 2e-5}
LOG_TOL = {"fp64": 1e-8, "fp32_split": 1e-5, "fp32": 1e-3}


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_02630_gb300 import qsvm
    qsvm.lib()
    return qsvm


def _dev(X):
    return torch.from_numpy(np.ascontiguousarray(X, dtype=np.float64)).cuda()


def _decode_fp64(buf, N, n, reps):
    """Site tensors A[i, k, sigma, t, u] and last-bond weights w[i, u] (None: the last bond is
    summed) from FP64 records (layouts of include/qsvm.h), with t = 2q + c, u = 2p + s.
    Block form (reps 1): a_0s[q][p] = A[s][2q][2p+s], then r; the rows with c = 1 are
    a_1s = r_s a_0s with r_0 = r, r_1 = conj(r).  Gauged form (reps 2): records k = 0..n of
    (alpha, beta) give a_0s = [[1, 1], [alpha, beta]] and a_1s = r'_s diag(1, -1) a_0s with
    r'_0 = alpha, r'_1 = beta; the virtual record n gives the weights of the last bond,
    w = (1, alpha_n, alpha_n, -alpha_n^2), and the state is 2^-n times the contraction, up to
    a global phase."""
    chi = 2 ** reps
    H = chi // 2
    A = np.zeros((N, n, 2, chi, chi), complex)
    w = None
    if reps == 3:
        # gauged, t = q + 4c and u = p + 4s with q = q1 + 2 q2: both blocks are
        # (-1)^{q1 q2} M[q1][p1] M[q2][p2] with M = [[1, 1], [alpha, beta]]; the c = 1 rows are
        # r'_s (-1)^{q2} times them; the virtual site weights the last bond
        raw = buf.cpu().numpy().view(np.complex128).reshape(N, n + 1, 2)
        al, be = raw[..., 0], raw[..., 1]
        def kr(a, b, q, p):
            m = lambda x, y: np.ones_like(a) if x == 0 else (a if y == 0 else b)
            return (-1) ** ((q & 1) * (q >> 1)) * m(q & 1, p & 1) * m(q >> 1, p >> 1)
        for s_ in range(2):
            rs = al[:, :n] if s_ == 0 else be[:, :n]
            for qq in range(4):
                for p in range(4):
                    v = kr(al[:, :n], be[:, :n], qq, p)
                    A[:, :, s_, qq, p + 4 * s_] = v
                    A[:, :, s_, qq + 4, p + 4 * s_] = rs * (1 - 2 * (qq >> 1)) * v
        an = al[:, n]
        w = np.zeros((N, 8), complex)
        for p in range(4):
            v0 = kr(an, an, p, 0)
            w[:, p] = v0
            w[:, p + 4] = an * (1 - 2 * (p >> 1)) * v0
        return A, w * 2.0 ** (-1.5 * n)
    if reps == 2:
        raw = buf.cpu().numpy().view(np.complex128).reshape(N, n + 1, 2)
        al, be = raw[..., 0], raw[..., 1]
        one = np.ones_like(al[:, :n])
        blocks = [np.stack([np.stack([one, one], -1), np.stack([al[:, :n], be[:, :n]], -1)], -2)] * 2
        for s_ in range(2):
            rs = al[:, :n] if s_ == 0 else be[:, :n]
            for qq in range(H):
                for p in range(H):
                    A[:, :, s_, 2 * qq, 2 * p + s_] = blocks[s_][:, :, qq, p]
                    A[:, :, s_, 2 * qq + 1, 2 * p + s_] = rs * (1 - 2 * qq) * blocks[s_][:, :, qq, p]
        an = al[:, n]
        w = np.stack([np.ones_like(an), an, an, -an * an], -1) * 2.0 ** (-n)
        return A, w
    raw = buf.cpu().numpy().view(np.complex128).reshape(N, n, 2 * H * H + 1)
    blocks = [raw[:, :, s * H * H:(s + 1) * H * H].reshape(N, n, H, H) for s in range(2)]
    r = raw[:, :, 2 * H * H]
    for s in range(2):
        rs = r if s == 0 else np.conj(r)
        for qq in range(H):
            for p in range(H):
                A[:, :, s, 2 * qq, 2 * p + s] = blocks[s][:, :, qq, p]
                A[:, :, s, 2 * qq + 1, 2 * p + s] = rs * blocks[s][:, :, qq, p]
    return A, w


def _mps_state(A, w=None):
    """Contract one point's site tensors A[k, sigma, t, u] to the 2^n state (qubit k = bit k);
    the last bond is summed, or weighted by w."""
    n, _, chi, _ = A.shape
    psi = np.zeros(2 ** n, complex)
    for s in range(2 ** n):
        v = np.zeros(chi, complex)
        v[0] = 1.0
        for k in range(n):
            v = v @ A[k, (s >> k) & 1]
        psi[s] = v.sum() if w is None else v @ w
    return psi


def _check(Kg, Ko, prec, what, LKg=None, LKo=None):
    err = np.max(np.abs(Kg - Ko))
    assert err <= TOL[prec], f"{what} {prec}: max|dK| = {err:.3e}"
    if LKg is not None:
        m = Ko > 1e-300
        if m.any():
            lerr = np.max(np.abs(LKg[m] - LKo[m]))
            assert lerr <= LOG_TOL[prec], f"{what} {prec}: max|dlnK| = {lerr:.3e}"
    return err


# ------------------------------------------------------------- builder -----
@pytest.mark.parametrize("reps", [1, 2, 3])
@pytest.mark.parametrize("n", [2, 3, 7, 10])
def test_build_mps_reproduces_state_vector(q, oracle, n, reps):
    X = inputs.uniform_features(3, n, 1000 + 10 * n + reps)
    buf = q.qsvm_build_mps(_dev(X), reps, "fp64")
    torch.cuda.synchronize()
    A, w = _decode_fp64(buf, 3, n, reps)
    for i in range(3):
        psi = _mps_state(A[i], None if w is None else w[i])
        ref = oracle.sv_state(X[i], reps)
        if w is not None:  # the gauged form fixes the state up to a global phase
            ph = np.vdot(psi, ref)
            assert abs(abs(ph) - 1.0) <= 1e-12
            psi = psi * ph / abs(ph)
        assert np.max(np.abs(psi - ref)) <= 1e-12


def test_build_mps_lowprec_formats(q):
    N, n, reps = 5, 33, 2
    X = inputs.mnist_like_features(N, n, 77)
    d = _dev(X)
    f64 = q.qsvm_build_mps(d, reps, "fp64").cpu().numpy().view(np.complex128).reshape(N, n + 1, 2)
    f32 = q.qsvm_build_mps(d, reps, "fp32").cpu().numpy().view(np.float32).reshape(N * n, 3, 2, 4)
    # the phases T^2, P^2, P^2 T^2 with theta_{k-1} = (pi - x_{k-1})(pi - x_k) (0 at site 0)
    theta = np.concatenate([np.zeros((N, 1)), (np.pi - X[:, :-1]) * (np.pi - X[:, 1:])], axis=1).reshape(-1)
    x = X.reshape(-1)
    want = np.stack([np.exp(-2j * theta), np.exp(-2j * x), np.exp(-2j * (x + theta))], axis=1)
    # gauged values: alpha_k = conj(V2^{k-1} V0^k), beta_k = conj(V2^{k-1}) V0^k (V2^{-1} = 1);
    # the virtual site n: alpha = beta = conj(V2^{n-1})
    V = want.reshape(N, n, 3)
    c = np.conj(np.concatenate([np.ones((N, 1)), V[:, :-1, 2]], axis=1))
    want_g = np.empty((N, n + 1, 2), complex)
    want_g[:, :n, 0] = c * np.conj(V[:, :, 0])
    want_g[:, :n, 1] = c * V[:, :, 0]
    want_g[:, n, 0] = want_g[:, n, 1] = np.conj(V[:, -1, 2])
    assert np.max(np.abs(f64 - want_g)) <= 1e-14

    def check_forms(a, b):  # a-form (re, im, -im, re); b-form (re, -im, im, re)
        re, im = a[..., 0], a[..., 1]
        assert np.array_equal(a[..., 2], -im) and np.array_equal(a[..., 3], re)
        assert np.array_equal(b[..., 0], re) and np.array_equal(b[..., 1], -im)
        assert np.array_equal(b[..., 2], im) and np.array_equal(b[..., 3], re)
        return re.astype(np.float64) + 1j * im.astype(np.float64)

    v32 = check_forms(f32[..., 0, :], f32[..., 1, :])
    for a, b in ((v32.real, want.real), (v32.imag, want.imag)):
        assert np.all(np.abs(a - b) <= np.abs(b) * 2.0 ** -24 + 1e-15)
    # split: two arrays (row-side a-forms, column-side b-forms) of n + 1 records of
    # (alpha, beta) x (hi, lo) entries, the same values as the FP64 records
    spl = q.qsvm_build_mps(d, reps, "fp32_split").cpu().numpy().view(np.float32).reshape(2, N, n + 1, 2, 2, 4)
    hi = check_forms(spl[0, :, :, :, 0, :], spl[1, :, :, :, 0, :])
    lo = check_forms(spl[0, :, :, :, 1, :], spl[1, :, :, :, 1, :])
    for part in (hi.real, hi.imag):
        assert np.array_equal(np.round(part * 2048) / 2048, part)
    assert np.max(np.abs(hi + lo - f64)) <= 2 ** -34


def test_build_mps_formats_reps3(q):
    """reps = 3: FP64 and split FP32 in the gauged form, whose records are those of reps = 2
    byte for byte (the reps = 3 gauge
    gives the signed Kronecker square of the same block), with alpha_k =
    exp(2 i (x_{k-1} + theta_{k-2} + theta_{k-1})) and beta_k with -theta_{k-1}."""
    N, n, reps = 3, 9, 3
    X = inputs.uniform_features(N, n, 91)
    d = _dev(X)
    f3 = q.qsvm_build_mps(d, reps, "fp64").cpu().numpy()
    f2 = q.qsvm_build_mps(d, 2, "fp64").cpu().numpy()
    assert f3.size == f2.size and np.array_equal(f3, f2)  # FP64: the gauged records of reps = 2
    s3 = q.qsvm_build_mps(d, reps, "fp32_split").cpu().numpy()
    s2 = q.qsvm_build_mps(d, 2, "fp32_split").cpu().numpy()
    assert s3.size == s2.size and np.array_equal(s3, s2)
    spl = s3.view(np.float32).reshape(2, N, n + 1, 2, 2, 4)
    th = np.concatenate([np.zeros((N, 1)), (np.pi - X[:, :-1]) * (np.pi - X[:, 1:]), np.zeros((N, 1))], axis=1)
    xp = np.concatenate([np.zeros((N, 1)), X], axis=1)      # x_{k-1} (0 at site 0)
    tp = np.concatenate([np.zeros((N, 1)), th[:, :-1]], axis=1)  # theta_{k-2}
    want = np.stack([np.exp(2j * (xp + tp + th)), np.exp(2j * (xp + tp - th))], axis=2)
    hi = spl[0, :, :, :, 0, 0] + 1j * spl[0, :, :, :, 0, 1].astype(np.float64)
    lo = spl[0, :, :, :, 1, 0] + 1j * spl[0, :, :, :, 1, 1].astype(np.float64)
    assert np.max(np.abs(hi.astype(np.complex128) + lo - want)) <= 2 ** -33


# ----------------------------------------------------------- small Grams ---
@pytest.mark.parametrize("prec", ["fp64", "fp32_split", "fp32"])
def test_gram_cfg0_vs_statevector(q, oracle, prec):
    X, _, n, reps = inputs.workload("cfg0_n8_r2_N16")
    Ko = oracle.sv_gram(X, reps)
    K, LK = q.gram(_dev(X), reps, prec, logK=True)
    Kg = K.cpu().numpy()
    _check(Kg, Ko, prec, "cfg0", LK.cpu().numpy(), np.log(np.maximum(Ko, 1e-320)))
    assert np.array_equal(Kg, Kg.T)


@pytest.mark.parametrize("prec", ["fp64", "fp32_split", "fp32"])
@pytest.mark.parametrize("reps", [1, 2, 3])
@pytest.mark.parametrize("N,n", [(1, 2), (17, 5), (100, 64), (37, 13)])
def test_gram_vs_mps_oracle(q, oracle, prec, reps, N, n):
    X = inputs.uniform_features(N, n, 7 * N + n + reps)
    Ko, LKo = oracle.mps_gram(X, reps)
    K, LK = q.gram(_dev(X), reps, prec, logK=True)
    Kg = K.cpu().numpy()
    _check(Kg, Ko, prec, f"gram N={N} n={n} reps={reps}", LK.cpu().numpy(), LKo)
    assert np.array_equal(Kg, Kg.T)
    assert q.qsvm_device_status() == 0


@pytest.mark.parametrize("prec", ["fp64", "fp32_split", "fp32"])
@pytest.mark.parametrize("reps", [1, 2, 3])
def test_cross_vs_mps_oracle(q, oracle, prec, reps):
    """Test x train with n_a != n_b, so a wrong column-side (b-form) offset in the
    two-array block formats (reps 1, 3) would show."""
    n = 64
    Xtr = inputs.uniform_features(53, n, 11)
    Xte = inputs.uniform_features(29, n, 12)
    Ko, LKo = oracle.mps_cross(Xte, Xtr, reps)
    K, LK = q.cross(_dev(Xte), _dev(Xtr), reps, prec, logK=True)
    _check(K.cpu().numpy(), Ko, prec, "cross", LK.cpu().numpy(), LKo)


def test_cross_leading_dimension(q, oracle):
    n, reps = 12, 2
    Xa, Xb = inputs.uniform_features(9, n, 3), inputs.uniform_features(21, n, 4)
    ma, mb = q.qsvm_build_mps(_dev(Xa), reps, "fp64"), q.qsvm_build_mps(_dev(Xb), reps, "fp64")
    big = torch.full((9, 40), -7.0, dtype=torch.float64, device="cuda")
    q.qsvm_kernel_cross(ma, 9, mb, 21, n, reps, "fp64", K=big[:, 5:26])
    B = big.cpu().numpy()
    Ko, _ = oracle.mps_cross(Xa, Xb, reps)
    assert np.max(np.abs(B[:, 5:26] - Ko)) <= 1e-10
    assert np.all(B[:, :5] == -7.0) and np.all(B[:, 26:] == -7.0)


@pytest.mark.parametrize("prec", ["fp64", "fp32_split", "fp32"])
@pytest.mark.parametrize("reps", [1, 2, 3])
def test_cross_row_slice(q, prec, reps):
    """mps + m * qsvm_mps_point_bytes as mps_a addresses points m.. of a buffer: the rows of
    that cross kernel equal rows m.. of the full one bit for bit (the row side reads only its
    own array, in every record format)."""
    na, nb, n, m = 37, 21, 9, 13
    Xa, Xb = inputs.uniform_features(na, n, 400 + reps), inputs.uniform_features(nb, n, 500 + reps)
    A, B = q.qsvm_build_mps(_dev(Xa), reps, prec), q.qsvm_build_mps(_dev(Xb), reps, prec)
    K, _ = q.qsvm_kernel_cross(A, na, B, nb, n, reps, prec)
    stride = q.qsvm_mps_point_bytes(n, reps, prec)
    assert stride % 16 == 0 and A.numel() == q.qsvm_mps_bytes(n, reps, na, prec)
    Ks, _ = q.qsvm_kernel_cross(A[m * stride:], na - m, B, nb, n, reps, prec)
    torch.cuda.synchronize()
    assert q.qsvm_device_status() == 0
    assert torch.equal(Ks, K[m:])


# ------------------------------------------------- n = 784 (paper's size) ---
@pytest.mark.parametrize("prec", ["fp64", "fp32_split"])
def test_gram_n784_mnist_like(q, oracle, prec):
    X = inputs.mnist_like_features(40, 784, 2)
    Ko, LKo = oracle.mps_gram(X, 2)
    K, LK = q.gram(_dev(X), 2, prec, logK=True)
    _check(K.cpu().numpy(), Ko, prec, "n784 gram", LK.cpu().numpy(), LKo)


@pytest.mark.parametrize("prec", ["fp64", "fp32_split", "fp32"])
def test_near_duplicates_n784(q, oracle, prec):
    # kernel values spread over (0, 1): the regime where |dK| <= 1e-6 is not vacuous
    base = inputs.mnist_like_features(24, 784, 21)
    pert = inputs.near_duplicates(base, 22)
    Ko, LKo = oracle.mps_cross(base, pert, 2)
    assert np.diag(Ko).min() < 0.9 and np.diag(Ko).max() > 0.99
    K, LK = q.cross(_dev(base), _dev(pert), 2, prec, logK=True)
    tol = {"fp64": 1e-10, "fp32_split": 1e-6, "fp32": 1e-4}[prec]
    err = np.max(np.abs(K.cpu().numpy() - Ko))
    assert err <= tol, f"{prec}: max|dK| = {err:.3e}"


@pytest.mark.parametrize("prec,reps", [("fp64", 2), ("fp32_split", 2), ("fp32_split", 3), ("fp64", 3), ("fp32", 2)])
def test_gram_near_duplicate_clusters_n784(q, oracle, prec, reps):
    """The symmetric Gram kernel (not the cross kernel) where |dK| <= 1e-6 bites: 24
    MNIST-like base rows with three perturbed copies each, shuffled, so that pairs with
    K in (0.1, 1) fall inside diagonal tiles (the kernel's masked half tile and mirror)
    and in off-diagonal tiles.  Every entry against the oracle, ln K where K > 1e-300,
    and the mirror bit-exact."""
    X, cl = inputs.near_duplicate_clusters(24, 4, 784, 40)
    N = X.shape[0]
    td = q.qsvm_gram_tile_dim(reps, prec)
    assert N > 2 * td
    Ko, LKo = oracle.mps_gram(X, reps)
    I, J = np.triu_indices(N, 1)
    big = Ko[I, J] > 0.1
    same_tile = (I // td) == (J // td)
    assert (big & same_tile).sum() >= 5 and (big & ~same_tile).sum() >= 20
    K, LK = q.gram(_dev(X), reps, prec, logK=True)
    Kg, LKg = K.cpu().numpy(), LK.cpu().numpy()
    assert q.qsvm_device_status() == 0
    assert np.array_equal(Kg, Kg.T) and np.array_equal(LKg, LKg.T)
    tol = 1e-4 if prec == "fp32" else TOL[prec]  # plain FP32's coherent rounding at n = 784
    err = np.max(np.abs(Kg - Ko))
    assert err <= tol, f"near-duplicate Gram {prec} reps={reps}: max|dK| = {err:.3e}"
    m = Ko > 1e-300
    assert np.max(np.abs(LKg[m] - LKo[m])) <= (1e-2 if prec == "fp32" else LOG_TOL[prec])
    # the informative entries on their own, in both kinds of tile
    for m in (big & same_tile, big & ~same_tile):
        assert np.max(np.abs(Kg[I[m], J[m]] - Ko[I[m], J[m]])) <= tol


def test_reps3_n784_logk(q, oracle):
    X = inputs.mnist_like_features(6, 784, 31)
    Ko, LKo = oracle.mps_gram(X, 3)
    K, LK = q.gram(_dev(X), 3, "fp64", logK=True)
    _check(K.cpu().numpy(), Ko, "fp64", "reps3 n784", LK.cpu().numpy(), LKo)
    L = LK.cpu().numpy()
    assert np.all(np.isfinite(L))
    assert np.max(np.abs(L - LKo)) <= 1e-8  # log K exact even where K underflows


# ----------------------------------------------------------- sharding ------
def test_gram_tile_ranges_compose(q):
    N, n, reps, prec = 70, 24, 2, "fp32_split"
    X = _dev(inputs.uniform_features(N, n, 5))
    mps = q.qsvm_build_mps(X, reps, prec)
    Kfull, _ = q.qsvm_kernel_gram(mps, N, n, reps, prec)
    Kpart = torch.full((N, N), float("nan"), dtype=torch.float64, device="cuda")
    for r in range(3):
        b, e = q.qsvm_gram_partition(N, reps, prec, 3, r)
        q.qsvm_kernel_gram_tiles(mps, N, n, reps, prec, b, e, Kpart)
    assert torch.equal(Kfull, Kpart)


# ------------------------------------------- full size, sampled (bench config) ---
def test_full_size_gram_sampled(q, oracle):
    """n = 784, reps = 2, N = 8192, split FP32, in the launch the bench times:
    bit-exact symmetry everywhere, and sampled entries against the oracle."""
    X, _, n, reps = inputs.workload("gram_n784_r2_N8192")
    N = X.shape[0]
    K, LK = q.gram(_dev(X), reps, "fp32_split", logK=True)
    torch.cuda.synchronize()
    assert q.qsvm_device_status() == 0
    assert torch.equal(K, K.T)
    rng = np.random.default_rng(0)
    di = rng.choice(N, 256, replace=False)
    ia = np.concatenate([di, rng.integers(0, N, 256)])
    ib = np.concatenate([di, rng.integers(0, N, 256)])
    Ko, LKo = oracle.mps_pairs(X, X, ia, ib, reps)
    Kg = K[torch.from_numpy(ia).cuda(), torch.from_numpy(ib).cuda()].cpu().numpy()
    LKg = LK[torch.from_numpy(ia).cuda(), torch.from_numpy(ib).cuda()].cpu().numpy()
    assert np.max(np.abs(Kg - Ko)) <= 1e-6
    m = Ko > 1e-300
    assert np.max(np.abs(LKg[m] - LKo[m])) <= 1e-5


def _sampled_pairs(N, seed, n_diag=256, n_rand=256, Nb=None):
    rng = np.random.default_rng(seed)
    di = rng.choice(N, min(n_diag, N), replace=False)
    ia = np.concatenate([di, rng.integers(0, N, n_rand)])
    ib = np.concatenate([di if Nb is None else rng.integers(0, Nb, di.size), rng.integers(0, Nb or N, n_rand)])
    return ia, ib


def test_full_size_gram_fp64_sampled(q, oracle):
    """The FP64 path at n = 784, reps = 2, N = 8192: bit-exact symmetry and |dK| <= 1e-10
    against the oracle on sampled entries (diagonal included)."""
    X, _, n, reps = inputs.workload("gram_n784_r2_N8192")
    K, LK = q.gram(_dev(X), reps, "fp64", logK=True)
    torch.cuda.synchronize()
    assert q.qsvm_device_status() == 0
    assert torch.equal(K, K.T)
    ia, ib = _sampled_pairs(X.shape[0], 1)
    Ko, LKo = oracle.mps_pairs(X, X, ia, ib, reps)
    Kg = K[torch.from_numpy(ia).cuda(), torch.from_numpy(ib).cuda()].cpu().numpy()
    LKg = LK[torch.from_numpy(ia).cuda(), torch.from_numpy(ib).cuda()].cpu().numpy()
    _check(Kg, Ko, "fp64", "full-size FP64 gram, sampled", LKg, LKo)  # |dK| <= 1e-10


def test_full_size_gram_reps3_sampled(q, oracle):
    """n = 784, reps = 3, N = 8192 (the four-thread engine, 8 x 8 tiles), split FP32:
    bit-exact symmetry and sampled entries against the oracle."""
    X, _, n, reps = inputs.workload("cfg4_n784_r3_N8192")
    K, LK = q.gram(_dev(X), reps, "fp32_split", logK=True)
    torch.cuda.synchronize()
    assert q.qsvm_device_status() == 0
    assert torch.equal(K, K.T)
    ia, ib = _sampled_pairs(X.shape[0], 2, 128, 128)
    Ko, LKo = oracle.mps_pairs(X, X, ia, ib, reps)
    Kg = K[torch.from_numpy(ia).cuda(), torch.from_numpy(ib).cuda()].cpu().numpy()
    LKg = LK[torch.from_numpy(ia).cuda(), torch.from_numpy(ib).cuda()].cpu().numpy()
    _check(Kg, Ko, "fp32_split", "full-size reps 3 gram, sampled", LKg, LKo)


@pytest.mark.parametrize("prec", ["fp32_split", "fp64"])
def test_full_size_cross_sampled(q, oracle, prec):
    """The 1024 x 2048 test x train kernel of the n = 784 MNIST-like workload (the launch
    the bench times) on sampled entries against the oracle."""
    Xtr, Xte, n, reps = inputs.workload("cfg2_n784_r2_N2048x1024")
    K, LK = q.cross(_dev(Xte), _dev(Xtr), reps, prec, logK=True)
    torch.cuda.synchronize()
    assert q.qsvm_device_status() == 0
    ia, ib = _sampled_pairs(Xte.shape[0], 3, 0, 512, Nb=Xtr.shape[0])
    Ko, LKo = oracle.mps_pairs(Xte, Xtr, ia, ib, reps)
    Kg = K[torch.from_numpy(ia).cuda(), torch.from_numpy(ib).cuda()].cpu().numpy()
    LKg = LK[torch.from_numpy(ia).cuda(), torch.from_numpy(ib).cuda()].cpu().numpy()
    _check(Kg, Ko, prec, "full-size cross, sampled", LKg, LKo)
