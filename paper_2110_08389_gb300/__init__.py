"""tweedmg: GB300-native geometric multigrid with tweed / wireframe smoothing.

Importing the package is cheap; the CUDA library is loaded on first use by
:mod:`paper_2110_08389_gb300.mg` and fails loudly when it is missing.
"""
__all__ = ["inputs", "mg"]
