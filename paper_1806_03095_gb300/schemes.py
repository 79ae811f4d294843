"""Coefficients of 2N-storage explicit Runge--Kutta schemes for dg_cns_lsrk_steps (Sec. 2.4: the
paper's integrator is a low-storage scheme of this form):

    dU <- A_i dU + dt L(U);   U <- U + B_i dU,   i = 1..s.

LSRK54: five stages, fourth order, Carpenter & Kennedy (1994), the scheme of dg_cns_rk_steps.
LSRK33: three stages, third order, Williamson (1980), the classic 2N scheme with rational
coefficients.  Both typed from their publications.  (The paper's own scheme, the seven-stage third
order scheme of Toulorge & Desmet, is not printed in it.)
"""

LSRK54 = (
    (0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
     -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0),
    (1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0, 1720146321549.0 / 2090206949498.0,
     3134564353537.0 / 4481467310338.0, 2277821191437.0 / 14882151754819.0),
)

LSRK33 = ((0.0, -5.0 / 9.0, -153.0 / 128.0), (1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0))

SCHEMES = {"lsrk54": LSRK54, "lsrk33": LSRK33}
