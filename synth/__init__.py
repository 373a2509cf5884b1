"""Seeded synthetic inputs for robust PCA, shared by the oracle, the tests and the benchmark.

This package only draws random problem instances and states the parameters the paper's
experiments pick for them (Section 3).  It holds none of the method's arithmetic: no
projection, threshold, factorisation or iteration of AccAltProj lives here.
"""
from .planted import PlantedInstance, planted_instance, paper_parameters, incoherence
from .video import VideoInstance, video_instance

__all__ = [
    "PlantedInstance",
    "planted_instance",
    "paper_parameters",
    "incoherence",
    "VideoInstance",
    "video_instance",
]
