"""FP64 CPU oracle for linearized plug-and-play ADMM with DSG-NLM.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package: only the
tests, the smoke check and the CPU-baseline leg of the benchmark do.  It is a
plain, slow, literal restatement of what the paper defines, in double precision,
and shares no code with the CUDA path (the only common module is the seeded input
generator ``synthetic``, which holds none of the method's arithmetic).

Modules
-------
``dsgnlm``   Sec. 3: NLM kernel (Eq. NLM), hat window (Eq. S1), symmetric
             normalisation (Eq. S2) iterated as symmetric Sinkhorn-Knopp, scaling
             and diagonal closure (Eq. S3), the explicit sparse W, and a literal
             transcription of Algorithm 2 for tiny images.
``forward``  Sec. 4.1 super-resolution model (blur + decimation, its adjoint, the
             gradient of Eq. dataterm, the Lipschitz constant) and Sec. 4.2
             single-photon model (Eq. obj, h and h'), plus the guide images.
``lpnp``     Algorithm 1 (linearized PnP-ADMM), residuals and PSNR.

Parity status of every function is listed in its module header; functions
without an independent pin say "parity unpinned".
"""
