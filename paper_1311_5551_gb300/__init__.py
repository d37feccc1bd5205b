"""GB300-native QED Monte-Carlo particle step (photon emission and pair production).

The compute path is a CUDA library (``csrc/``, sm_103a) behind a C ABI (``include/qed.h``);
``qed`` is its thin ctypes binding.  Importing this package does not load the library:
``qed.lib()`` does, and fails loudly when the compiled extension is missing.
"""
