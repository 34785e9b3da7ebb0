"""GB300-native all-pairs Smith-Waterman read distances (arxiv 1803.02272, section 2.2).

Importing the package does not load the CUDA library; `paper_1803_02272_gb300.gbd`
does, and fails loudly when it is missing.
"""
__all__ = ["synth"]
