"""GB300 (sm_103a) library for one SDPD time step with a Metropolised
Shardlow-like fluctuation/dissipation sweep (Faure & Stoltz).

The compute path is the CUDA library built from ``csrc/`` (C ABI declared in
``include/sdpd.h``); ``sdpd`` is its ctypes binding and ``inputs`` the seeded
synthetic initial states.
"""

__all__ = ["inputs", "sdpd", "build"]
