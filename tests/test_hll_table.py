"""The library's HLL wave-speed table (rt_wave_table: analytic Jacobian, characteristic
cubic in extended precision) against the oracle's (complex-step Jacobian, numpy
eigenvalues).  Host computation on both sides: no GPU needed."""
import numpy as np

from oracle import m1_eigen
from paper_2302_12727_gb300 import RT_WAVE_NF, RT_WAVE_NTH, rt_wave_table


def test_library_wave_table_matches_oracle():
    lmax, lmin = rt_wave_table()
    omax, omin = m1_eigen.default_table()
    assert lmax.shape == (RT_WAVE_NF, RT_WAVE_NTH) == omax.shape
    # the oracle's eigen-solver is accurate to ~5e-14 on these non-normal Jacobians
    np.testing.assert_allclose(lmax, omax, rtol=0, atol=1e-13)
    np.testing.assert_allclose(lmin, omin, rtol=0, atol=1e-13)
