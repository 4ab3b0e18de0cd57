"""1D quadrature and Lagrange tables on [0,1], and a plain LU with partial pivoting.

Every routine here works elementwise on numpy arrays or Python floats and states
its evaluation order, because the graph decisions downstream are reproduced bit
for bit by an independent implementation.
"""
import math
import numpy as np

NEWTON_STEPS = 100   # fixed Newton step count for Gauss-Legendre roots


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [0,1] (paper Sec. 2: volume and face integrals
    by Gauss-Legendre quadrature).  Returns (nodes ascending, weights).

    Roots of P_n on [-1,1] by Newton's method from x_i = cos(pi (i + 0.75) / (n + 0.5)),
    i = 0..n-1, exactly NEWTON_STEPS steps, with the three-term recurrence
    P_k = ((2k-1) x P_{k-1} - (k-1) P_{k-2}) / k and P_n' = n (x P_n - P_{n-1}) / (x x - 1).
    Mapped: t = 0.5 (1 - x), w = 1 / ((1 - x x) P_n'(x) P_n'(x)).
    """
    if n < 1:
        raise ValueError("n >= 1")
    nodes, weights = [], []
    for i in range(n):
        x = math.cos(math.pi * (i + 0.75) / (n + 0.5))
        dp = 0.0
        for _ in range(NEWTON_STEPS + 1):
            p0, p1 = 1.0, x
            for k in range(2, n + 1):
                p0, p1 = p1, ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k
            dp = n * (x * p1 - p0) / (x * x - 1.0)
            if _ < NEWTON_STEPS:
                x = x - p1 / dp
        nodes.append(0.5 * (1.0 - x))
        weights.append(1.0 / ((1.0 - x * x) * dp * dp))
    return np.array(nodes), np.array(weights)


def gll_nodes(p):
    """Gauss-Lobatto-Legendre nodes of order p on [0,1] (the DG nodal basis, Sec. 2:
    u_m(x_n) = delta_mn; node choice is a reading, the paper only says Lagrangian)."""
    if p == 1:
        return np.array([0.0, 1.0])
    if p == 2:
        return np.array([0.0, 0.5, 1.0])
    if p == 3:
        a = 1.0 / math.sqrt(5.0)
        return np.array([0.0, 0.5 * (1.0 - a), 0.5 * (1.0 + a), 1.0])
    raise ValueError("DG order p must be 1, 2 or 3")


def equispaced_nodes(r):
    """Geometry control-point nodes a/r, a = 0..r (Q_r map of eq. 1)."""
    return np.array([a / r for a in range(r + 1)], dtype=np.float64)


def lagrange(nodes, j, x):
    """l_j(x) = prod_{k != j} (x - n_k)/(n_j - n_k), multiplied left to right from 1.0."""
    v = 1.0
    for k in range(len(nodes)):
        if k != j:
            v = v * ((x - nodes[k]) / (nodes[j] - nodes[k]))
    return v


def lagrange_deriv(nodes, j, x):
    """l_j'(x) = sum_{k != j} [1/(n_j - n_k)] prod_{l != j,k} (x - n_l)/(n_j - n_l);
    the outer sum from 0.0 in increasing k, each product left to right."""
    d = 0.0
    for k in range(len(nodes)):
        if k == j:
            continue
        t = 1.0 / (nodes[j] - nodes[k])
        for l in range(len(nodes)):
            if l != j and l != k:
                t = t * ((x - nodes[l]) / (nodes[j] - nodes[l]))
        d = d + t
    return d


def lu_factor(A):
    """Doolittle LU with partial pivoting, plain loops, in a copy of A (n x n).

    Pivot = first row index i >= k with the largest |A[i][k]|; full rows are swapped.
    For i > k: l = A[i][k] / A[k][k]; A[i][j] = A[i][j] - l * A[k][j] for j > k.
    Returns (LU, perm) with perm[k] = original row now in position k.
    """
    A = [list(map(float, row)) for row in np.asarray(A, dtype=np.float64)]
    n = len(A)
    perm = list(range(n))
    for k in range(n):
        p, best = k, abs(A[k][k])
        for i in range(k + 1, n):
            if abs(A[i][k]) > best:
                p, best = i, abs(A[i][k])
        if best == 0.0:
            raise np.linalg.LinAlgError("singular matrix in lu_factor")
        if p != k:
            A[k], A[p] = A[p], A[k]
            perm[k], perm[p] = perm[p], perm[k]
        for i in range(k + 1, n):
            l = A[i][k] / A[k][k]
            A[i][k] = l
            for j in range(k + 1, n):
                A[i][j] = A[i][j] - l * A[k][j]
    return A, perm


def lu_solve(LU, perm, b):
    """Solve with lu_factor's output: y = P b; forward (unit L), backward (U), plain loops,
    inner sums in increasing column order."""
    n = len(LU)
    y = [float(b[perm[i]]) for i in range(n)]
    for i in range(n):
        for j in range(i):
            y[i] = y[i] - LU[i][j] * y[j]
    for i in range(n - 1, -1, -1):
        for j in range(i + 1, n):
            y[i] = y[i] - LU[i][j] * y[j]
        y[i] = y[i] / LU[i][i]
    return np.array(y)


def lu_solve_dense(A, b):
    """A x = b by lu_factor/lu_solve (b may be a matrix: columns solved one by one)."""
    LU, perm = lu_factor(A)
    b = np.asarray(b, dtype=np.float64)
    if b.ndim == 1:
        return lu_solve(LU, perm, b)
    return np.stack([lu_solve(LU, perm, b[:, c]) for c in range(b.shape[1])], axis=1)
