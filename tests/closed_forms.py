"""Closed-form values of tiny TPFA networks, solved by hand (no oracle code)."""


def checkerboard_closed_form(a, b, lx, lz):
    """Load along z of the 2 x 2 checkerboard [[a, b], [b, a]] in the x-z plane.

    Hand solution of the four-cell network of Sec. 2.2 (A = (0,0) kappa a,
    B = (1,0) kappa b, C = (0,1) kappa b, D = (1,1) kappa a; p_in = 1 at
    k = -1/2, p_out = 0).  A half-turn about y maps the medium to itself and
    swaps the two Dirichlet faces, so p_C = 1 - p_B and p_D = 1 - p_A; the
    balances at A and B are then a 2 x 2 system, solved by Cramer's rule.
    Returns (K[x][z], K[z][z]) of the off-diagonal definition (mean x-face
    flux times L^z / dp) and of the outflow formula.
    """
    hx, hz = lx / 2.0, lz / 2.0
    m = 2.0 * a * b / (a + b)
    tx, tz = m / hx ** 2, m / hz ** 2            # harmonic faces of kappa~
    ba, bb = 2.0 * a / hz ** 2, 2.0 * b / hz ** 2  # Dirichlet faces 2 kappa~^z
    a11, a12, r1 = tx + tz + ba, tz - tx, tz + ba
    a21, a22, r2 = tz - tx, tx + tz + bb, tz + bb
    det = a11 * a22 - a12 * a21
    pa = (r1 * a22 - a12 * r2) / det
    pb = (a11 * r2 - a21 * r1) / det
    mean_vx = 2.0 * tx * hx * (pa - pb) / 4.0     # two x faces, four cells
    kxz = lz * mean_vx
    kzz = lz * hz * (bb * (1.0 - pb) + ba * (1.0 - pa)) / 2.0
    return kxz, kzz
