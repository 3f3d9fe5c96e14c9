"""CPU oracle for the pWave++ decode path (test infrastructure only).

This package is a plain, slow, obviously-correct CPU implementation of what
the CUDA library computes, written from the paper ("Efficient Learned Wavelet
Image and Video Coding", pWave++ / pMCTF):

* lifting.py  - CNN lifting wavelet transform (Section 3.1, Fig. 2), float
                and integer-rounded, plus the temporal (MCTF-style) lifting
                of Section 3.3 with identity motion.
* context.py  - ConvLSTM context prediction and the four-step context fusion
                nets (Section 3.2, Figs. 3-5), and the autoregressive LL model.
* entropy.py  - entropy parameters -> table indices, and the deterministic
                FP32 Laplace CDF table bank (Section 3.1: Laplace model).
* rans.py     - interleaved rANS coder standing in for the paper's adaptive
                arithmetic coder.
* codec.py    - colour conversion, quantiser, coding order, bitstream
                container, encode / decode of images and GOPs.
* blob.py     - reader of the weight-blob file format.

It is test infrastructure: only the tests, the smoke entry point and the
benchmark's CPU-baseline leg may import it. The product path (the CUDA
library and its Python binding) never imports or calls anything here, and
nothing here imports the product.

Floating-point work is FP64, except the entropy-parameter index decision and
the CDF table bank, whose definition is FP32 (encoder and decoder must agree
bit for bit, so the precision is part of the format).

Parity status per function is stated in each module header; functions whose
only pin is their own definition say "parity unpinned".
"""
