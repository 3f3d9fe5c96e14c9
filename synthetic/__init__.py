"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This package holds input generators only: images, video frames, request
streams and random-init weight blobs. It contains none of the codec's
arithmetic (no transform, no context model, no entropy coding), so both sides
of every parity test can draw their inputs from here without sharing code.
"""
from .images import (gray_sinusoids, rgb_natural, video_gop, lossless_blobs,
                     request_stream)
from .weights import ModelConfig, random_model, pack_blob, tensor_specs

__all__ = ["gray_sinusoids", "rgb_natural", "video_gop", "lossless_blobs",
           "request_stream", "ModelConfig", "random_model", "pack_blob",
           "tensor_specs"]
