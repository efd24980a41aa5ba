"""Conversion between oracle H^2 matrices and the flat factor layout of h2_import/h2_export
(ranks of every box; leaf bases; transfer matrices; lower far couplings; lower near
blocks; all column-major FP64 -- see include/h2.h).  The converters live in the oracle
package (oracle.h2.factor_arrays / from_factor_arrays); these are the names the tests use.
"""
from oracle.h2 import factor_arrays as oracle_to_import        # noqa: F401
from oracle.h2 import from_factor_arrays as import_to_oracle   # noqa: F401
