"""Host helpers of the photo-ionisation sink (rt_cross_section, rt_blackbody_groups,
rt_photon_number_to_luminosity: the library's own quadrature) against the oracle
(scipy quadrature) and the thesis's printed group luminosities.  No GPU needed."""
import math

import numpy as np
import pytest

from oracle import photo
from paper_2302_12727_gb300 import RTError, rt_blackbody_groups, rt_cross_section, rt_photon_number_to_luminosity

EDGES = ([3.288e15, 5.945e15, 13.157e15, math.inf], [3.288e15 * k for k in range(1, 11)] + [math.inf],
         [5e14, 3.288e15, 1e16, 2e16])


def test_library_group_averages_match_oracle():
    for e in EDGES:
        for T in (3e4, 1e5):
            a = rt_blackbody_groups(T, e)
            b = photo.group_averages(T, e)
            for x, y in zip(a, b):
                np.testing.assert_allclose(x, y, rtol=1e-9, atol=1e-12 * np.abs(y).max())
            np.testing.assert_allclose(rt_photon_number_to_luminosity(T, 5e48, e),
                                       photo.number_to_luminosity(T, 5e48, e), rtol=1e-9)
    for j, s in enumerate(photo.SPECIES):
        for E in (10.0, 13.6, 24.6, 30.0, 54.5, 100.0, 1000.0):
            assert rt_cross_section(j, E) == pytest.approx(photo.cross_section(s, E), rel=1e-13, abs=0.0)


def test_library_reproduces_the_printed_luminosities():
    """Iliev test 2 of the thesis: 5e48 photons/s of a 1e5 K blackbody in three groups
    (1.764e4, 3.631e4, 8.037e3 L_sun, with L_sun = 3.826e33 erg/s)."""
    L = rt_photon_number_to_luminosity(1e5, 5e48, EDGES[0]) / 3.826e33
    np.testing.assert_allclose(L, [1.764e4, 3.631e4, 8.037e3], rtol=6e-4)


def test_invalid_arguments_are_rejected():
    with pytest.raises(RTError):
        rt_blackbody_groups(1e5, [3e15, 2e15])
    with pytest.raises(RTError):
        rt_blackbody_groups(-1.0, [3e15, 4e15])
    with pytest.raises(RTError):
        rt_cross_section(3, 20.0)
