"""Solver settings that depend on the strength of the convection.

At a thermal expansion coefficient alpha of 1e6 (the paper's strongly convective cases, Sec. 6 and 7)
the temperature transport is convection-dominated along the buoyancy direction z, and the multigrid
levels below the finest smooth with the z-line block-Jacobi smoother (NC_SMOOTH_ZLINE) and damping
omega = 0.7. Measured on the GB300 at 80 x 80 x 160 and alpha = 1e6: the cylinder's state solve takes
46 instead of 191 Krylov iterations, the cavity's 85 instead of 130, and every case is faster. At
alpha = 1e4 the z-line smoother leaves the Krylov count unchanged and costs time, so below the
threshold the library defaults (2x2 block Jacobi, omega = 0.9) stay.
"""

from ._abi import NC_SMOOTH_ZLINE

ZLINE_FROM_ALPHA = 1e6


def solver_settings(alpha):
    """nc_params overrides for a problem at thermal expansion coefficient alpha (empty below the
    threshold). The smoother is fixed when a problem is created, so a problem that climbs an alpha
    ladder (warm starts, Sec. 5.4) takes the settings of the ladder's target."""
    if alpha >= ZLINE_FROM_ALPHA:
        return {"mg_smoother": NC_SMOOTH_ZLINE, "omega": 0.7}
    return {}
