"""Seeded synthetic inputs shared by the CUDA-path tests, the oracle tests and the benchmark.

This module holds no arithmetic of the method (no filter, interpolation or discretisation
of the paper): it only draws designs and request streams with NumPy's PCG64 generator so
that the oracle and the CUDA library see identical bytes.

Design families (element arrays ordered i + nx*(j + ny*k), gamma = 1 solid, 0 fluid):

* ``filtered_random``: i.i.d. N(0, 1) per element, smoothed with a cone kernel of radius
  1.5 elements (weights max(0, 1.5 - distance)), min-max mapped to [0, 1]; with a target
  volume fraction V the field is shifted by c (bisection) so that mean(clip(x + c, 0, 1)) = V.
* ``fin_plates``: 8 vertical plates normal to x, each 2 elements thick, evenly spaced, full
  y extent, from the top of the heated layers up to z = 0.75 of the height, plus N(0, 0.05)
  noise, clipped to [0, 1].
* ``request_stream``: Poisson arrivals (rate 20/s), grid edge uniform over
  {32, 48, 64, 96, 128}, buoyancy factor log-uniform in [1e3, 1e5], half state-only and half
  state+adjoint, each with its own filtered-random design seed.
* ``filtered_random_torch``: the filtered_random recipe in torch on a device, seeded by torch's
  own generator (used where hundreds of designs must be drawn quickly, e.g. the serving stream).
"""

from .designs import filtered_random, filtered_random_torch, fin_plates, request_stream  # noqa: F401
