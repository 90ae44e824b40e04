"""B300-native rerandomization balance checks (FastRerandomize hot path, arXiv 2501.07642).

The compute path is the CUDA library libfrr.so behind include/frr.h;
``paper_2501_07642_b300.frr`` is its thin Python binding.
"""
