"""Level-symmetric (LQn) discrete-ordinate sets.

The paper (Sec. 2, after eq. 2) only requires omega_d > 0 and sum omega_d = 4*pi;
its results use level-symmetric S2/S4 sets.  The sets here follow the standard
LQn construction: direction cosines mu_i^2 = mu_1^2 + (i-1) * 2(1 - 3 mu_1^2)/(N-2),
octant points = index triples (i,j,k) with i+j+k = N/2 + 2, point weights shared
by each permutation class.  mu_1 and the class weights are the published LQn
table values (7 digits); the weights are normalised so each octant sums to 1.
"""
import numpy as np

# N -> (mu_1, {sorted 1-based level-index triple: point weight within an octant})
_LQN = {
    2: (0.5773502691896257, {(1, 1, 1): 1.0}),
    4: (0.3500212, {(1, 1, 2): 1.0 / 3.0}),
    6: (0.2666355, {(1, 1, 3): 0.1761263, (1, 2, 2): 0.1572071}),
    8: (0.2182179, {(1, 1, 4): 0.1209877, (1, 2, 3): 0.0907407, (2, 2, 2): 0.0925926}),
    12: (0.1672126, {(1, 1, 6): 0.0707626, (1, 2, 5): 0.0558811, (1, 3, 4): 0.0373377,
                     (2, 2, 4): 0.0502819, (2, 3, 3): 0.0258513}),
}


def level_symmetric(N, dim):
    """Return (omega [M,3] float64, w [M] float64) for the S_N level-symmetric set.

    dim == 3: all 8 octants, M = N(N+2), w = (pi/2) * octant point weight.
    dim == 2: the xi > 0 hemisphere only (the problem is z-invariant), M = N(N+2)/2,
              w = pi * octant point weight (each point stands for its mirror image).
    Directions are ordered octant by octant (signs (+,+,+), (-,+,+), (+,-,+), (-,-,+),
    then z<0 for 3D), points within an octant by their index triple.
    sum(w) == 4*pi up to rounding.
    """
    if N not in _LQN:
        raise ValueError(f"level-symmetric S{N} not tabulated (have {sorted(_LQN)})")
    mu1, table = _LQN[N]
    n = N // 2
    if N == 2:
        mus = np.array([mu1])
    else:
        mus = np.sqrt(np.array([mu1 * mu1 + i * 2.0 * (1.0 - 3.0 * mu1 * mu1) / (N - 2) for i in range(n)]))
    pts = [(i, j, k) for k in range(1, n + 1) for j in range(1, n + 1) for i in range(1, n + 1)
           if i + j + k == n + 2]
    pw = np.array([table[tuple(sorted(p))] for p in pts], dtype=np.float64)
    tot = 0.0
    for x in pw:             # left to right in point order (a fixed summation order)
        tot = tot + float(x)
    pw = pw / tot
    base = np.array([[mus[i - 1], mus[j - 1], mus[k - 1]] for (i, j, k) in pts], dtype=np.float64)
    if dim == 3:
        signs = [(sx, sy, sz) for sz in (1, -1) for sy in (1, -1) for sx in (1, -1)]
        scale = np.pi / 2.0
    elif dim == 2:
        signs = [(sx, sy, 1) for sy in (1, -1) for sx in (1, -1)]
        scale = np.pi
    else:
        raise ValueError("dim must be 2 or 3")
    om = np.concatenate([base * np.array(s, dtype=np.float64) for s in signs], axis=0)
    w = np.concatenate([pw * scale for _ in signs])
    return np.ascontiguousarray(om), np.ascontiguousarray(w)
