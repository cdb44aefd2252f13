"""ORACLE -- test infrastructure only.

A plain double-precision CPU restatement of the periodisation method
(arXiv 1310.4374) plus an independent Ewald sum.  Only the tests, the smoke
check and the benchmark's CPU-baseline leg may use it; the product path never
imports it and shares no code with it.
"""
