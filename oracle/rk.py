"""Low-storage explicit Runge--Kutta time stepping (oracle; test infrastructure only).

Sec. 2.4 integrates dU/dt = L(U, t) with an explicit s-stage scheme in Butcher
form and low-storage variants that keep one vector besides U_n and U_{n+1}.
The workloads here use the five-stage fourth-order 2N-storage scheme of
Carpenter & Kennedy (1994, NASA TM-109112, solution 3), coefficients typed
from that publication:

    dU <- A_i dU + dt L(U, t + C_i dt);   U <- U + B_i dU,   i = 1..5.

Pinned by tests/test_oracle_rk_diag.py: the Butcher tableau derived from (A, B)
satisfies all eight order-<=4 conditions, c_i = sum_j a_ij reproduces C, and
y' = lambda y shows order 4.

The general 2N stage (any coefficients) is lsrk_step; the second scheme here is
Williamson's (1980) three-stage third-order 2N scheme, whose rational
coefficients are typed from that publication (pinned by the four order-<=3
conditions, its failure of order 4, and y' = lambda y showing order 3).
"""
from fractions import Fraction

LSRK54_A = (
    Fraction(0),
    Fraction(-567301805773, 1357537059087),
    Fraction(-2404267990393, 2016746695238),
    Fraction(-3550918686646, 2091501179385),
    Fraction(-1275806237668, 842570457699),
)
LSRK54_B = (
    Fraction(1432997174477, 9575080441755),
    Fraction(5161836677717, 13612068292357),
    Fraction(1720146321549, 2090206949498),
    Fraction(3134564353537, 4481467310338),
    Fraction(2277821191437, 14882151754819),
)
LSRK54_C = (
    Fraction(0),
    Fraction(1432997174477, 9575080441755),
    Fraction(2526269341429, 6820363962896),
    Fraction(2006345519317, 3224310063776),
    Fraction(2802321613138, 2924317926251),
)

LSRK33_A = (Fraction(0), Fraction(-5, 9), Fraction(-153, 128))
LSRK33_B = (Fraction(1, 3), Fraction(15, 16), Fraction(8, 15))
LSRK33_C = (Fraction(0), Fraction(1, 3), Fraction(3, 4))

STAGES = 5
A = tuple(float(a) for a in LSRK54_A)
B = tuple(float(b) for b in LSRK54_B)
C = tuple(float(c) for c in LSRK54_C)


def butcher_from_2n(Acoef, Bcoef):
    """Butcher (a, b) of a 2N scheme.

    With k_j the stage derivatives, dU_i = dt sum_{j<=i} (prod_{l=j+1}^{i} A_l) k_j
    and U^(i) = U_n + sum_{m<=i} B_m dU_m, so
    a_{i+1, j} = sum_{m=j}^{i} B_m prod_{l=j+1}^{m} A_l and b_j = a_{s+1, j}.
    """
    s = len(Acoef)
    a = [[Fraction(0)] * s for _ in range(s + 1)]
    for i in range(s):          # row i+1 (0-based: stage i+1 uses U^(i))
        for j in range(i + 1):
            tot = Fraction(0)
            for m in range(j, i + 1):
                prod = Fraction(1)
                for l in range(j + 1, m + 1):
                    prod *= Acoef[l]
                tot += Bcoef[m] * prod
            a[i + 1][j] = tot
    return [row[:] for row in a[:s]], a[s]


def step(Lfun, U, dt, t, dU=None):
    """One 2N-storage RK(5,4) step of dU/dt = Lfun(U, t); returns U_{n+1}."""
    dU = U * 0.0 if dU is None else dU
    for i in range(STAGES):
        dU = A[i] * dU + dt * Lfun(U, t + C[i] * dt)
        U = U + B[i] * dU
    return U


def lsrk_step(Lfun, U, dt, t, Acoef, Bcoef, Ccoef):
    """One step of the 2N scheme with stage coefficients (A_i, B_i, C_i) of dU/dt = Lfun(U, t)."""
    dU = U * 0.0
    for Ai, Bi, Ci in zip(Acoef, Bcoef, Ccoef):
        dU = float(Ai) * dU + dt * Lfun(U, t + float(Ci) * dt)
        U = U + float(Bi) * dU
    return U
