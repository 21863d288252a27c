"""Pins of the oracle's learned-sensor pieces: BF16 rounding against a library
conversion, features and network on closed-form cases, and the plain-detector
labels on a step."""
import numpy as np
import pytest

from paper_2305_00762_gb300 import cases as C


@pytest.fixture(scope="module")
def OS(oracle_mod):
    import oracle.sensor as S
    return S


def test_bf16_round_matches_torch(OS):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=5000).astype(np.float32),
                        (rng.normal(size=5000) * 1e-4).astype(np.float32)])
    # exact ties: low 16 bits = 0x8000 with even and odd kept bit
    ties = (np.arange(64, dtype=np.uint32) << 16 | 0x3F808000).view(np.float32)
    x = np.concatenate([x, ties, -ties])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(OS.bf16_round(x), ref)


def test_features_of_a_ramp(oracle_mod, OS):
    """rho = 1 + b x, p uniform: f_k = dx_k b h / (2|b h| + 1e-3), p part 0."""
    O = oracle_mod
    n, b = 16, 0.3
    xc, h = C.centres(n, 0.0, 1.0)
    X, _ = np.meshgrid(xc, xc)
    Q = C.prim_to_cons(1 + b * X, 0 * X, 0 * X, 1 + 0 * X, 1.4)
    cfg = O.Config(n, n, h, h, 1.4, 0.0, 0.72, (1, 1, 0, 0))
    f = OS.features(cfg, Q).reshape(n, n, 50)
    cell = f[8, 8]
    bh = np.float32(b * h)
    for k in range(25):
        dx = k % 5 - 2
        assert abs(cell[k] - dx * bh / (2 * bh + 1e-3)) < 1e-5
    assert np.abs(cell[25:]).max() < 1e-6


def test_network_closed_form(OS):
    """W1 = [I; 0] on the first 32 inputs, W2 = I, w3 = 1, zero biases:
    z = sum_n relu(bf16(relu(x_n))) for n < 32."""
    W1 = np.zeros((50, 32), np.float32)
    W1[:32, :32] = np.eye(32)
    w = np.concatenate([W1.ravel(), np.zeros(32), np.eye(32, dtype=np.float32).ravel(), np.zeros(32),
                        np.ones(32), [0.0]]).astype(np.float32)
    x = np.random.default_rng(1).normal(size=(10, 50)).astype(np.float32) * 0.3
    xb = OS.bf16_round(x)
    z = OS.bf16_round(np.maximum(xb[:, :32], 0)).sum(axis=1)
    p = OS.forward(x, w)
    assert np.allclose(p, 1 / (1 + np.exp(-z)), atol=1e-6)
    assert list(OS.decision([0.1, 0.3, 0.5, 0.7, 0.9])) == [0, 2, 2, 2, 1]


def test_labels_at_a_step(oracle_mod):
    """A density jump between columns s-1 and s: psi < 0.5 exactly on the
    four columns s-2..s+1 (Eq. detector), in every row."""
    O = oracle_mod
    n, s = 24, 11
    rho = np.where(np.arange(n)[None, :] >= s, 0.4, 1.0) * np.ones((n, 1))
    z = np.zeros_like(rho)
    Q = C.prim_to_cons(rho, z, z, 1 + z, 1.4)
    cfg = O.Config(n, n, 0.1, 0.1, 1.4, 0.0, 0.72, (1, 1, 0, 0))
    lab = O.trouble_labels(cfg, Q)
    cols = np.nonzero(lab[0])[0]
    assert list(cols) == [s - 2, s - 1, s, s + 1]
    assert np.all(lab == lab[0])


def test_psi_min_at_a_step_and_flat(oracle_mod, OS):
    """Eq. detector by hand: on flat data a = b = 0 and psi = eps/eps = 1;
    beside a density step 1 -> 0.4 (stencil 1, 1, 1, 0.4, 0.4 centred on the
    last 1) a = 0, b = 0.6 + 0.6, psi = eps / (1.44 + eps). Labels are exactly
    psi_min < 1/2, and the soft target is 1/2 there, monotone in psi."""
    O = oracle_mod
    n, s = 24, 11
    rho = np.where(np.arange(n)[None, :] >= s, 0.4, 1.0) * np.ones((n, 1))
    z = np.zeros_like(rho)
    Q = C.prim_to_cons(rho, z, z, 1 + z, 1.4)
    cfg = O.Config(n, n, 0.1, 0.1, 1.4, 0.0, 0.72, (1, 1, 0, 0))
    psi = O.psi_min(cfg, Q)
    eps = 0.9 * 0.5 / (1 - 0.9 * 0.5) * 1e-6
    assert np.all(psi[:, :s - 3] == 1.0) and np.all(psi[:, s + 3:] == 1.0)
    assert psi[5, s - 1] == pytest.approx(eps / (1.44 + eps), rel=1e-12)
    assert np.array_equal(O.trouble_labels(cfg, Q), (psi < 0.5).astype(np.uint8))
    Qr = C.kelvin_helmholtz(32, np.random.default_rng(9)).Q
    cr = O.Config(32, 32, 1 / 32, 1 / 32, 1.4, 0.0, 0.72, (0, 0, 0, 0))
    pr = O.psi_min(cr, Qr)
    assert np.array_equal(O.trouble_labels(cr, Qr), (pr < 0.5).astype(np.uint8))
    t = OS.soft_target(np.array([0.0, 0.5 - 0.8 * OS.TAU, 0.5, 0.5 + 0.8 * OS.TAU, 1.0]))
    assert t[0] == 255 and t[-1] == 0 and t[2] == 128
    assert 0.3 * 255 < t[3] < t[2] < t[1] < 0.7 * 255 + 1


def test_features_at_equals_features(oracle_mod, OS):
    O = oracle_mod
    c = C.kelvin_helmholtz(24, np.random.default_rng(2), ny=20)
    cfg = O.Config(c.nx, c.ny, c.dx, c.dy, c.gamma, c.mu, c.Pr, c.bc)
    full = OS.features(cfg, c.Q).reshape(c.ny, c.nx, 50)
    rng = np.random.default_rng(3)
    rows, cols = rng.integers(0, c.ny, 40), rng.integers(0, c.nx, 40)
    assert np.array_equal(OS.features_at(cfg, c.Q, rows, cols), full[rows, cols])


def test_direction_flags_rule(OS):
    """Decision table of the learned sensor's per-direction flags."""
    p = np.array([0.1, 0.1, 0.5, 0.5, 0.5, 0.9, 0.9, 0.9, 0.9])
    tx = np.array([1, 0, 1, 0, 0, 1, 0, 0, 1], bool)
    ty = np.array([1, 0, 0, 1, 0, 0, 1, 0, 1], bool)
    fx, fy = OS.direction_flags(p, tx, ty)
    assert list(fx) == [0, 0, 1, 0, 0, 1, 0, 1, 1]
    assert list(fy) == [0, 0, 0, 1, 0, 0, 1, 1, 1]
