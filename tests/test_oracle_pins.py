"""Pins for the reference oracle against facts fixed outside the oracle.

Each check ties the oracle to something other than itself:

* closed forms (Bloch-sphere rotations under u(t) = exp(-i t P / 2), the
  rotation definition of Sec. 3.3);
* an independent dense brute force (numpy Kronecker products and
  ``scipy.linalg.expm`` of Pauli matrices) for n <= 4, including gradients by
  the exact parameter-shift rule on that dense code;
* invariants: norm preservation, |E| <= 1, 2*pi periodicity, light-cone zeros
  of the hardware-efficient ansatz, truncation to the light cone;
* central finite differences of the oracle's own loss (a different code path
  from its adjoint sweep).

Each catches a plausible slip: a wrong RZ sign or half-angle fails the closed
forms and the dense check; a transposed qubit order fails the d=1 closed form
(which singles out qubit 0) and the dense check; a dropped factor 2 in the
seed (Eq. 4) or a wrong dL/dE weighting fails parameter shift and FD; a wrong
dagger in the adjoint update (Eq. 2) fails parameter shift.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import oracle as orc
from paper_2603_02804_gb300 import workloads

PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)
PI = np.eye(2, dtype=complex)
PAULI_MAT = {0: PI, 1: PX, 2: PY, 3: PZ}
ROT_GEN = {orc.RX: PX, orc.RY: PY, orc.RZ: PZ}


# ---------------------------------------------------------------- dense code
def _embed(n, q, m):
    """Operator m on qubit q (qubit q = bit q of the index, LSB = qubit 0)."""
    return np.kron(np.eye(1 << (n - 1 - q)), np.kron(m, np.eye(1 << q)))


def _dense_rot(kind, t):
    return scipy.linalg.expm(-0.5j * t * ROT_GEN[kind])


def _dense_two(n, kind, c, t):
    dim = 1 << n
    U = np.zeros((dim, dim), dtype=complex)
    for x in range(dim):
        if kind == orc.CZ:
            U[x, x] = -1.0 if ((x >> c) & 1 and (x >> t) & 1) else 1.0
        else:  # CNOT
            y = x ^ (1 << t) if (x >> c) & 1 else x
            U[y, x] = 1.0
    return U


def dense_unitary(circ, theta):
    n = circ.n
    U = np.eye(1 << n, dtype=complex)
    for kind, q0, q1, p in circ.gates:
        if kind in (orc.CZ, orc.CNOT):
            G = _dense_two(n, kind, q0, q1)
        else:
            G = _embed(n, q0, _dense_rot(kind, float(theta[p])))
        U = G @ U
    return U


def dense_encode(n, x):
    psi = np.zeros(1 << n, dtype=complex)
    psi[0] = 1.0
    for q in range(n):
        psi = _embed(n, q, _dense_rot(orc.RY, float(x[q]))) @ psi
    return psi


def dense_observable(n, letters):
    O = np.eye(1, dtype=complex)
    for q in reversed(range(n)):  # highest qubit is the leftmost Kronecker factor
        O = np.kron(O, PAULI_MAT[int(letters[q])])
    return O


def dense_E(circ, theta, x, obs):
    O = dense_observable(circ.n, orc.pauli_letters(circ.n, obs))
    U = dense_unitary(circ, theta)
    out = []
    for row in np.atleast_2d(x):
        psi = U @ dense_encode(circ.n, row)
        out.append(np.real(np.vdot(psi, O @ psi)))
    return np.array(out)


def dense_param_shift(circ, theta, x, obs):
    """Exact parameter-shift rule for exp(-i t P/2) gates, per sample."""
    theta = np.asarray(theta, dtype=np.float64)
    g = np.zeros((len(np.atleast_2d(x)), circ.n_params))
    for p in range(circ.n_params):
        tp = theta.copy(); tp[p] += np.pi / 2
        tm = theta.copy(); tm[p] -= np.pi / 2
        g[:, p] = 0.5 * (dense_E(circ, tp, x, obs) - dense_E(circ, tm, x, obs))
    return g


def random_circuit(n, n_gates, rng, shared_params=0, kinds=(orc.RX, orc.RY, orc.RZ, orc.CZ, orc.CNOT)):
    """Random gate list. Each rotation gets its own parameter unless
    shared_params > 0, in which case indices are drawn from that many."""
    rows = []
    n_params = 0
    for _ in range(n_gates):
        k = int(rng.choice(kinds))
        if k in (orc.CZ, orc.CNOT):
            if n < 2:
                continue
            a, b = rng.choice(n, size=2, replace=False)
            rows.append((k, int(a), int(b), -1))
        else:
            if shared_params:
                p = int(rng.integers(shared_params))
            else:
                p = n_params
                n_params += 1
            rows.append((k, int(rng.integers(n)), -1, p))
    n_params = shared_params or n_params
    return orc.Circuit(n=n, gates=np.array(rows, dtype=np.int32).reshape(-1, 4), n_params=n_params)


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("t", [0.0, 0.3, 1.0, np.pi / 2, 2.5, np.pi, 4.0, 5.9])
def test_ry_encoding_gives_cos(t):
    # <Z> after RY(t)|0> = cos t
    c = orc.hea(1, 0)
    E = orc.expectation(c, np.zeros(0), np.array([[t]]), "Z")
    assert abs(E[0] - np.cos(t)) < 1e-14


@pytest.mark.parametrize("t", [0.2, 1.7, 3.3, 6.0])
def test_single_rotations_closed_forms(t):
    g = lambda k, q=0: orc.Circuit(1, np.array([[k, q, -1, 0]], np.int32), 1)
    th = np.array([t])
    zero = np.array([[0.0]])
    plus = np.array([[np.pi / 2]])  # RY(pi/2)|0> = |+>
    assert abs(orc.expectation(g(orc.RY), th, zero, "Z")[0] - np.cos(t)) < 1e-14
    assert abs(orc.expectation(g(orc.RX), th, zero, "Z")[0] - np.cos(t)) < 1e-14
    assert abs(orc.expectation(g(orc.RX), th, zero, "Y")[0] + np.sin(t)) < 1e-14
    assert abs(orc.expectation(g(orc.RZ), th, zero, "Z")[0] - 1.0) < 1e-14
    assert abs(orc.expectation(g(orc.RZ), th, plus, "X")[0] - np.cos(t)) < 1e-14
    assert abs(orc.expectation(g(orc.RZ), th, plus, "Y")[0] - np.sin(t)) < 1e-14


@pytest.mark.parametrize("n", [1, 2, 5, 7])
def test_hea_depth1_closed_form(n):
    """d=1, O=Z_0: the CZ chain and the last RZ commute with Z_0, so only
    RY(x0), RZ(a0), RY(b0) on qubit 0 matter:
    E = cos x0 cos b0 - sin x0 cos a0 sin b0."""
    rng = np.random.default_rng(7 + n)
    c = orc.hea(n, 1)
    theta = rng.uniform(0, 2 * np.pi, c.n_params)
    x = rng.uniform(0, np.pi, (3, n))
    grad, E = orc.gradient(c, theta, x, "Z", per_sample=True)
    a0, b0 = theta[0], theta[1]
    for s in range(3):
        x0 = x[s, 0]
        assert abs(E[s] - (np.cos(x0) * np.cos(b0) - np.sin(x0) * np.cos(a0) * np.sin(b0))) < 1e-13
        expect = np.zeros(c.n_params)
        expect[0] = np.sin(x0) * np.sin(a0) * np.sin(b0)
        expect[1] = -np.cos(x0) * np.sin(b0) - np.sin(x0) * np.cos(a0) * np.cos(b0)
        assert np.max(np.abs(grad[s] - expect)) < 1e-13


# ---------------------------------------------------------------- dense brute force
@pytest.mark.parametrize("n,d", [(1, 2), (2, 1), (3, 2), (4, 2)])
@pytest.mark.parametrize("obs", ["Z", "X", "Y", "ZZ", "XYZI", "IXYZ", "YY"])
def test_hea_matches_dense(n, d, obs):
    obs = obs[:n].ljust(n, "I")
    rng = np.random.default_rng(100 * n + d)
    c = orc.hea(n, d, "ring" if n > 2 else "chain")
    theta = rng.uniform(0, 2 * np.pi, c.n_params)
    x = rng.uniform(0, np.pi, (2, n))
    E = orc.expectation(c, theta, x, obs)
    assert np.max(np.abs(E - dense_E(c, theta, x, obs))) < 1e-12


@pytest.mark.parametrize("seed", range(6))
def test_random_circuits_match_dense_and_param_shift(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 5))
    c = random_circuit(n, 14, rng)
    theta = rng.uniform(-np.pi, 3 * np.pi, c.n_params)
    x = rng.uniform(0, np.pi, (3, n))
    obs = "".join(rng.choice(list("IXYZ"), size=n))
    E_dense = dense_E(c, theta, x, obs)
    dLdE = rng.normal(size=3)
    grad, E = orc.gradient(c, theta, x, obs, dLdE=dLdE, per_sample=True, block=int(rng.integers(1, 9)))
    assert np.max(np.abs(E - E_dense)) < 1e-12
    ps = dense_param_shift(c, theta, x, obs) * dLdE[:, None]
    assert np.max(np.abs(grad - ps)) < 1e-12
    gsum, _ = orc.gradient(c, theta, x, obs, dLdE=dLdE, per_sample=False)
    assert np.max(np.abs(gsum - ps.sum(0))) < 1e-12


@pytest.mark.parametrize("seed", range(3))
def test_shared_parameters_match_dense_fd(seed):
    """A parameter used by several gates: the adjoint sums every occurrence.
    Checked against central differences of the dense brute force."""
    rng = np.random.default_rng(50 + seed)
    n = 3
    c = random_circuit(n, 16, rng, shared_params=4)
    theta = rng.uniform(0, 2 * np.pi, c.n_params)
    x = rng.uniform(0, np.pi, (2, n))
    grad, _ = orc.gradient(c, theta, x, "ZXY")
    h = 1e-5
    for p in range(c.n_params):
        tp = theta.copy(); tp[p] += h
        tm = theta.copy(); tm[p] -= h
        fd = (dense_E(c, tp, x, "ZXY").sum() - dense_E(c, tm, x, "ZXY").sum()) / (2 * h)
        assert abs(fd - grad[p]) < 1e-8


def test_init_state_path_matches_dense():
    rng = np.random.default_rng(5)
    n = 3
    c = orc.hea(n, 2)
    theta = rng.uniform(0, 2 * np.pi, c.n_params)
    psi0 = workloads.draw_state(2, n, 9).astype(np.complex128)
    U = dense_unitary(c, theta)
    O = dense_observable(n, orc.pauli_letters(n, "XZY"))
    ref = [np.real(np.vdot(U @ p, O @ (U @ p))) for p in psi0]
    E = orc.expectation(c, theta, None, "XZY", init_states=psi0)
    assert np.max(np.abs(E - ref)) < 1e-12


# ---------------------------------------------------------------- invariants
def test_norm_and_bounds():
    rng = np.random.default_rng(3)
    c = orc.hea(6, 4)
    theta = rng.uniform(0, 2 * np.pi, c.n_params)
    for row in rng.uniform(0, np.pi, (4, 6)):
        psi = orc.final_state(c, theta, row)
        assert abs(np.vdot(psi, psi).real - 1.0) < 1e-13
    E = orc.expectation(c, theta, rng.uniform(0, np.pi, (16, 6)), "ZXYZII")
    assert np.all(np.abs(E) <= 1 + 1e-13)


def test_two_pi_periodicity():
    rng = np.random.default_rng(4)
    c = orc.hea(5, 3)
    theta = rng.uniform(0, 2 * np.pi, c.n_params)
    x = rng.uniform(0, np.pi, (3, 5))
    E0 = orc.expectation(c, theta, x, "Z")
    for p in rng.choice(c.n_params, 6, replace=False):
        t2 = theta.copy(); t2[p] += 2 * np.pi  # U -> -U: global phase
        assert np.max(np.abs(orc.expectation(c, t2, x, "Z") - E0)) < 1e-12


@pytest.mark.parametrize("n,d", [(6, 3), (7, 2), (5, 5)])
def test_light_cone_zeros_and_truncation(n, d):
    """For O = Z_0, rotations on qubit q of layer l lie outside the backward
    light cone when q > d-1-l, and the final RZ on qubit 0 commutes with Z_0."""
    rng = np.random.default_rng(11 * n + d)
    c = orc.hea(n, d)
    theta = rng.uniform(0, 2 * np.pi, c.n_params)
    x = rng.uniform(0, np.pi, (2, n))
    grad, E = orc.gradient(c, theta, x, "Z", per_sample=True)
    g = grad.reshape(2, d, n, 3)
    for l in range(d):
        for q in range(n):
            if q > d - 1 - l:
                assert np.max(np.abs(g[:, l, q, :])) < 1e-13
    assert np.max(np.abs(g[:, d - 1, 0, 2])) < 1e-13
    # inside the light cone the gradient is generically nonzero
    assert np.max(np.abs(g[:, 0, 0, 1])) > 1e-6
    # truncation: E on n qubits equals E on min(n, d) qubits
    m = min(n, d)
    ct = orc.hea(m, d)
    tt = theta.reshape(d, n, 3)[:, :m, :].reshape(-1)
    Et = orc.expectation(ct, tt, x[:, :m], "Z")
    assert np.max(np.abs(E - Et)) < 1e-12


def test_mirror_light_cone_high_qubit():
    """O = Z_{n-1}: the mirrored statement, q < n-d+l has zero gradient."""
    n, d = 7, 3
    rng = np.random.default_rng(21)
    c = orc.hea(n, d)
    theta = rng.uniform(0, 2 * np.pi, c.n_params)
    x = rng.uniform(0, np.pi, (2, n))
    obs = "I" * (n - 1) + "Z"
    grad, _ = orc.gradient(c, theta, x, obs, per_sample=True)
    g = grad.reshape(2, d, n, 3)
    for l in range(d):
        for q in range(n):
            if q < n - d + l:
                assert np.max(np.abs(g[:, l, q, :])) < 1e-13


# ---------------------------------------------------------------- gradients
def test_parameter_shift_on_oracle_energy():
    rng = np.random.default_rng(8)
    c = orc.hea(6, 3, "ring")
    theta = rng.uniform(0, 2 * np.pi, c.n_params)
    x = rng.uniform(0, np.pi, (2, 6))
    grad, _ = orc.gradient(c, theta, x, "IXYZIX")
    for p in rng.choice(c.n_params, 12, replace=False):
        tp = theta.copy(); tp[p] += np.pi / 2
        tm = theta.copy(); tm[p] -= np.pi / 2
        ps = 0.5 * (orc.expectation(c, tp, x, "IXYZIX") - orc.expectation(c, tm, x, "IXYZIX")).sum()
        assert abs(grad[p] - ps) < 1e-12


def test_mse_finite_difference():
    """Central FD (h = 1e-3) of L = mean (E - y)^2 against the adjoint gradient.
    Truncation error is about h^2/6 |L'''|, below 1e-7 here."""
    w = workloads.Workload("fd", 6, 4, 16, "mse", "Z", (1, 2, 3))
    theta, x, y = workloads.make_inputs(w)
    theta = theta.astype(np.float64)
    c = orc.hea(w.n, w.d)
    E = orc.expectation(c, theta, x, "Z")
    grad, _ = orc.gradient(c, theta, x, "Z", dLdE=orc.mse_dLdE(E, y))
    h = 1e-3
    for p in workloads.draw_fd_params(c.n_params, 16, 4):
        tp = theta.copy(); tp[p] += h
        tm = theta.copy(); tm[p] -= h
        fd = (orc.mse_loss(orc.expectation(c, tp, x, "Z"), y)
              - orc.mse_loss(orc.expectation(c, tm, x, "Z"), y)) / (2 * h)
        assert abs(fd - grad[p]) < 1e-6


def test_block_size_does_not_change_gradient():
    rng = np.random.default_rng(12)
    c = orc.hea(5, 4)
    theta = rng.uniform(0, 2 * np.pi, c.n_params)
    x = rng.uniform(0, np.pi, (3, 5))
    ref, _ = orc.gradient(c, theta, x, "ZZ", per_sample=True, block=len(c.gates))
    for blk in (1, 7, 33):
        g, _ = orc.gradient(c, theta, x, "ZZ", per_sample=True, block=blk)
        assert np.max(np.abs(g - ref)) < 1e-13


def test_threads_do_not_change_result():
    rng = np.random.default_rng(13)
    c = orc.hea(6, 3)
    theta = rng.uniform(0, 2 * np.pi, c.n_params)
    x = rng.uniform(0, np.pi, (9, 6))
    g1, e1 = orc.gradient(c, theta, x, "Z", threads=1)
    g4, e4 = orc.gradient(c, theta, x, "Z", threads=4)
    assert np.array_equal(g1, g4) and np.array_equal(e1, e4)


def test_amplitude_parallel_mode_matches_serial():
    """With fewer samples than threads the oracle splits its amplitude loops
    over the threads (n >= 17). Pinned against closed forms there, and against
    the one-thread run, which differs only in the order of the final sums."""
    n = 17
    c = orc.hea(n, 1)
    rng = np.random.default_rng(17)
    theta = rng.uniform(0, 2 * np.pi, c.n_params)
    x = rng.uniform(0, np.pi, (2, n))
    g_par, e_par = orc.gradient(c, theta, x, "Z", per_sample=True, threads=4)
    a0, b0 = theta[0], theta[1]
    for s in range(2):
        x0 = x[s, 0]
        assert abs(e_par[s] - (np.cos(x0) * np.cos(b0) - np.sin(x0) * np.cos(a0) * np.sin(b0))) < 1e-13
        expect = np.zeros(c.n_params)
        expect[0] = np.sin(x0) * np.sin(a0) * np.sin(b0)
        expect[1] = -np.cos(x0) * np.sin(b0) - np.sin(x0) * np.cos(a0) * np.cos(b0)
        assert np.max(np.abs(g_par[s] - expect)) < 1e-13
    c2 = orc.hea(n, 2)
    theta2 = rng.uniform(0, 2 * np.pi, c2.n_params)
    g1, e1 = orc.gradient(c2, theta2, x[:1], "ZIX", per_sample=True, threads=1)
    g4, e4 = orc.gradient(c2, theta2, x[:1], "ZIX", per_sample=True, threads=4)
    assert np.max(np.abs(g1 - g4)) < 1e-12 and np.max(np.abs(e1 - e4)) < 1e-12
    assert np.max(np.abs(g1)) > 1e-3  # a non-trivial gradient
