"""GB300-native molecular-dynamics hot path after Colberg & Hoefling (arXiv:0912.3824).

Importing the package loads nothing compiled.  ``paper_0912_3824_gb300.md``
binds the CUDA shared library (it raises if the library is missing);
``paper_0912_3824_gb300.synth`` holds the seeded input generators.
"""
__all__ = ["md", "synth"]
