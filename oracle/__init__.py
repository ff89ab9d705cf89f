"""FP64 CPU oracle for the Helmholtz / U-Net hot path.

TEST INFRASTRUCTURE ONLY.  Imported by tests/, the smoke check and the
benchmark's CPU-baseline and reference legs; never by the product path, and
sharing no code with the CUDA library (only the seeded input generators in
paper_2203_11025_gb300/synth.py feed both).
"""
