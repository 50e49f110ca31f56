"""Block-filtered exchange-correlation quadrature on GB300 (sm_103a).

The compute path lives in ``libkldi.so`` (C ABI in ``include/kldi.h``); the
Python module ``kldi`` is a ctypes binding with the same entry-point names.
"""
__all__ = ["kldi"]
