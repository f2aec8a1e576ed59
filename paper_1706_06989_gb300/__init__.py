"""GB300 (sm_103a) implementation of the angular-momentum-conserving Cartesian
fast multipole method (Marcello 2017, built on Dehnen 2000).

The compute path is the C-ABI library ``libamfmm.so`` built from ``csrc/``;
``paper_1706_06989_gb300.fmm`` is its thin ctypes binding.  Importing this
package loads nothing; the binding loads the library on first use and raises
if it is missing.
"""
__all__ = ["fmm", "ics"]
