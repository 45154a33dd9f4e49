"""Complex moment-based interior SVD (Imakura & Sakurai) on GB300.

The compute path lives in the C-ABI library ``libcmsvd.so`` (hand-written
sm_103a CUDA). ``binding`` marshals arguments to it; ``synth`` builds seeded
synthetic inputs.
"""
