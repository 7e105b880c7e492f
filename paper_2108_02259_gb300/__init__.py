"""libapiccontact: the APIC augury contact step (arXiv 2108.02259) on GB300.

Importing the package loads nothing; ``paper_2108_02259_gb300.apic`` loads the
CUDA library on first use and raises if it has not been built.
"""
