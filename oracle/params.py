"""Problem description for the oracle (test infrastructure only).

Readings of the paper fixed here:
* The xy box is [0, Lx) x [0, Ly) and Lx is the full period, so h = Lx/Nx and
  k = 2*pi*n/Lx.  (Sec. II writes the box as [-L, L] with k = n*pi/L; Table III pairs
  L = 128.8 R_h with Nxy = 150 and m = 4, which only gives the Table II radius if L is the
  full period.)
* The grid spacing is the same in x and y (Sec. II footnote: square boxes); the kernel
  support is alpha = m*h/2 for both the monopole and the dipole kernel (Sec. III.E).
"""

from dataclasses import dataclass

FREE = "free"
BOTTOM_WALL = "bottom_wall"
SLIT = "slit"
MODES = (FREE, BOTTOM_WALL, SLIT)


def table1(m):
    """Table I (force and torque, M & D): (R_h/h, beta_M/m, beta_D/m) for m = 5, 6."""
    return {5: (1.560, 1.305, 2.232), 6: (1.731, 1.327, 2.216)}[m]


def table2(m):
    """Table II (force only, M): (R_h/h, beta_M/m) for m = 4, 5, 6."""
    return {4: (1.205, 1.785), 5: (1.344, 1.886), 6: (1.554, 1.714)}[m]


@dataclass(frozen=True)
class Params:
    """Box, wall mode, grid and ES-kernel parameters of one mobility problem.

    mode  : 'free' (open in z, Sec. III), 'bottom_wall' (no-slip wall at zmin, open above;
            Sec. III.B) or 'slit' (no-slip walls at zmin and zmax; Appendix A with l0 = lH = 0).
    nz    : number of Chebyshev nodes on [zmin, zmax] including both endpoints (Sec. III.D).
    m_M, beta_M / m_D, beta_D : ES support width in grid cells and shape parameter of the
            monopole / dipole kernels (Sec. III.E, Eq. 54); alpha = m*h/2.
    eta   : viscosity (Eq. 4).
    slip_bottom, slip_top : slip lengths l0 at zmin and lH at zmax (Appendix A, Eq. A1); 0 is a
            no-slip wall.  The bottom-wall geometry takes l0 only; the open geometry neither.
    uw_bottom, uw_top : uniform tangential wall velocities (u^W, v^W) at zmin and zmax (Eq. A1;
            the paper allows any smooth u^W(x, y), only uniform ones are modelled here).
    """

    Lx: float
    Ly: float
    zmin: float
    zmax: float
    mode: str
    nx: int
    ny: int
    nz: int
    m_M: int
    beta_M: float
    m_D: int = 0
    beta_D: float = 0.0
    eta: float = 1.0
    slip_bottom: float = 0.0
    slip_top: float = 0.0
    uw_bottom: tuple = (0.0, 0.0)
    uw_top: tuple = (0.0, 0.0)

    def __post_init__(self):
        if self.mode not in MODES:
            raise ValueError(f"unknown wall mode {self.mode!r}")
        if self.nx < 2 or self.ny < 2 or self.nz < 3:
            raise ValueError("grid too small")
        if abs(self.Lx / self.nx - self.Ly / self.ny) > 1e-12 * (self.Lx / self.nx):
            raise ValueError("the grid spacing must be the same in x and y")
        if not self.zmax > self.zmin:
            raise ValueError("zmax must exceed zmin")
        if not (self.slip_bottom >= 0.0 and self.slip_top >= 0.0):
            raise ValueError("slip lengths must be non-negative")
        top_wall = self.mode == SLIT
        bottom_wall = self.mode in (BOTTOM_WALL, SLIT)
        if not bottom_wall and (self.slip_bottom or any(self.uw_bottom)):
            raise ValueError("no bottom wall to carry slip or a wall velocity")
        if not top_wall and (self.slip_top or any(self.uw_top)):
            raise ValueError("no top wall to carry slip or a wall velocity")

    @property
    def h(self):
        return self.Lx / self.nx

    @property
    def H(self):
        return self.zmax - self.zmin

    @property
    def alpha_M(self):
        return 0.5 * self.m_M * self.h

    @property
    def alpha_D(self):
        return 0.5 * self.m_D * self.h
