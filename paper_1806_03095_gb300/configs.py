"""Named workloads (Taylor--Green vortex of Sec. 4.2.1; turbulent channel of Sec. 4.3.1).

Sizes follow the benchmark configurations: TGV 8^3 / 64^3 k=3, 40^3 k=5,
24^3 k=4 on [-pi, pi]^3; channel 2 pi x 2 x pi with 32^3 cells, k=3.
Quadrature: nq_conv = floor(3k/2)+1 (3/2-rule), nq_visc = k+1.
"""
import math

PI = math.pi


def tgv(N, k, precision=0, kernel=2):
    return dict(name="tgv%d_k%d" % (N, k), ncells=(N, N, N), lo=(-PI,) * 3, hi=(PI,) * 3, periodic=(1, 1, 1),
                k=k, nq_conv=(3 * k) // 2 + 1, nq_visc=k + 1, Re=1600.0, Ma=0.1, Pr=0.71, gamma=1.4, R=287.0,
                u_mach=0.0, body_force=(0.0, 0.0, 0.0), mapping=0, map_param=0.0, precision=precision,
                kernel=kernel, u_max=1.0, h_min=2 * PI / N, Cr=0.4, D=0.02)


def channel_h_min(N, C=1.8):
    """Minimum vertex distance of the stretched channel grid: the wall-adjacent cell height."""
    y0 = math.tanh(C * (2.0 * 0.0 - 1.0)) / math.tanh(C)
    y1 = math.tanh(C * (2.0 * (1.0 / N) - 1.0)) / math.tanh(C)
    return min(y1 - y0, 2 * PI / N, PI / N)


def channel(N=32, k=3, precision=1, kernel=2, mapping=1):
    return dict(name="channel%d_k%d" % (N, k), ncells=(N, N, N), lo=(0.0, -1.0, 0.0), hi=(2 * PI, 1.0, PI),
                periodic=(1, 0, 1), k=k, nq_conv=(3 * k) // 2 + 1, nq_visc=k + 1, Re=180.0, Ma=0.1, Pr=0.71,
                gamma=1.4, R=287.0, u_mach=18.3, body_force=(1.0, 0.0, 0.0), mapping=mapping, map_param=1.8,
                precision=precision, kernel=kernel, u_max=18.3, h_min=channel_h_min(N), Cr=0.4, D=0.02)


WORKLOADS = {
    "tgv8_k3": lambda **kw: tgv(8, 3, **kw),
    "tgv64_k3": lambda **kw: tgv(64, 3, **kw),
    "tgv48_k3": lambda **kw: tgv(48, 3, **kw),
    "tgv32_k3": lambda **kw: tgv(32, 3, **kw),
    "tgv40_k5": lambda **kw: tgv(40, 5, **kw),
    "tgv24_k4": lambda **kw: tgv(24, 4, **kw),
    "tgv16_k15": lambda **kw: tgv(16, 15, **kw),
    "tgv8_k15": lambda **kw: tgv(8, 15, **kw),
    "channel32_k3": lambda **kw: channel(32, 3, **kw),
}


def make_context(cfg, device=None):
    from .api import DGCNS
    return DGCNS(cfg["ncells"], cfg["lo"], cfg["hi"], cfg["periodic"], cfg["k"], cfg["nq_conv"], cfg["nq_visc"],
                 gamma=cfg["gamma"], Pr=cfg["Pr"], Re=cfg["Re"], Ma=cfg["Ma"], R=cfg["R"], u_mach=cfg["u_mach"],
                 body_force=cfg["body_force"], precision=cfg["precision"], kernel=cfg["kernel"],
                 mapping=cfg["mapping"], map_param=cfg["map_param"], deform=cfg.get("deform", 0.0),
                 geometry=cfg.get("geometry", 0), device=device)


def time_step(cfg, h_min=None):
    """Eq. TimeStepRestrictions_Compressible with e = 1.5, f = 3, nu = mu / rho0 = U0 L / Re."""
    from .api import cfl_dt
    h = cfg["h_min"] if h_min is None else h_min
    nu = 1.0 / cfg["Re"] if cfg["u_mach"] == 0 else 1.0 / cfg["Re"]
    return cfl_dt(cfg["k"], h, cfg["u_max"], cfg["Ma"], Cr=cfg["Cr"], D=cfg["D"], nu=nu)
