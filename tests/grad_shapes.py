"""Clouds of the gradient pins: a flat film, the same cloud tilted, and a film
on a spherical cap (film rows whose neighbours lie off their tangent plane),
each with a 3D cube.  Inputs only: generator calls, no method arithmetic."""
from paper_2405_13165_gb300 import clouds as C

SHAPES = ("flat", "tilted", "curved")


def shape(name, dx=0.05):
    """(cloud, dx) of one of SHAPES."""
    if name == "flat":
        return C.cube_on_sheet(dx, cube=8 * dx, sheet=20 * dx), dx     # 512 + 384 particles
    if name == "tilted":
        return C.rotated(C.cube_on_sheet(dx, cube=8 * dx, sheet=20 * dx), (1.0, 0.4, 0.2), 0.6), dx
    if name == "curved":
        cap = C.curved_film(dx, 11 * dx, 14 * dx)
        cube = C.cube_on_sheet(dx, cube=5 * dx, sheet=7 * dx)
        cube.pos_h[:, 2] += 10 * dx    # lifted clear of the cap
        return C.concat([cap, cube]), dx
    raise ValueError(name)
