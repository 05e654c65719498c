"""GB300 (sm_103a) DSG-NLM denoiser and linearized plug-and-play ADMM.

The compute path is the CUDA library ``lib/libdsgnlm.so`` (C ABI in
``include/dsgnlm.h``); ``dsgnlm`` is its thin PyTorch binding and ``pipeline``
strings the calls together for the experiments of the paper.
"""
