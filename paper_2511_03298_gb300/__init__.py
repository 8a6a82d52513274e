"""GB300-native KScaNN query path (arXiv 2511.03298).

The compute lives in the CUDA library built from csrc/ (loaded lazily by
`paper_2511_03298_gb300.ksc`); `synth` holds the seeded synthetic inputs.
"""
__all__ = ["ksc", "synth"]
