"""Dense-matrix helpers for the tests (textbook definitions, n <= 8)."""
import numpy as np

I2 = np.eye(2, dtype=complex)
SX = np.array([[0, 1], [1, 0]], dtype=complex)
SY = np.array([[0, -1j], [1j, 0]], dtype=complex)
SZ = np.array([[1, 0], [0, -1]], dtype=complex)
HD = np.array([[1, 1], [1, -1]], dtype=complex) / np.sqrt(2)
SD = np.array([[1, 0], [0, 1j]], dtype=complex)


def single(n, q, U):
    """U on qubit q; qubit q is index bit q (qubit 0 least significant)."""
    M = np.ones((1, 1), dtype=complex)
    for k in reversed(range(n)):
        M = np.kron(M, U if k == q else I2)
    return M


def pauli(n, x, z):
    M = np.ones((1, 1), dtype=complex)
    for k in reversed(range(n)):
        b = ((x >> k) & 1) + 2 * ((z >> k) & 1)
        M = np.kron(M, [I2, SX, SZ, SY][b])
    return M


def cnot(n, c, t):
    N = 1 << n
    M = np.zeros((N, N), dtype=complex)
    for v in range(N):
        M[v ^ (((v >> c) & 1) << t), v] = 1
    return M


def cz(n, c, t):
    N = 1 << n
    return np.diag([(-1.0) ** (((v >> c) & 1) & ((v >> t) & 1)) for v in range(N)]).astype(complex)


def gate(n, g):
    k, a, b = g
    if k == "H":
        return single(n, a, HD)
    if k == "S":
        return single(n, a, SD)
    if k == "CNOT":
        return cnot(n, a, b)
    if k == "CZ":
        return cz(n, a, b)
    raise ValueError(k)


def circuit(n, gates):
    """Unitary of a gate list in application order (first gate acts first)."""
    C = np.eye(1 << n, dtype=complex)
    for g in gates:
        C = gate(n, g) @ C
    return C


def hamiltonian(n, x, z, c):
    H = np.zeros((1 << n, 1 << n), dtype=complex)
    for a, b, v in zip(x, z, c):
        H += v * pauli(n, int(a), int(b))
    return H
