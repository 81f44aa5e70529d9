"""CPU oracle for the FEnc^2 encrypted-convolution hot path.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
reference that the CUDA library is checked against.  Only tests/, the smoke
check in __graft_entry__ and the CPU-baseline leg of bench.py may import it;
the library never does.  It shares no code, header, table or constant generator
with the CUDA path; the only module both sides read is the seeded input
generator in workloads/, which holds no arithmetic of the method.

Modules:
  _core / ckks_core.c  modular arithmetic, NTT, sampling, encode/decode (C)
  ckks                 RNS-CKKS scheme operations, rotation (Eq. 1), rescale
  fragment             conv-aware fragment encoding (Algorithm 1)
  counts               rotation-complexity model (Eq. 3 - Eq. 8)
  plain                FP64 plaintext network (Eq. 2 and the layers around it)
  henn                 encrypted conv / activation / pool / FC / AAC
  boot                 the ciphertext refresh (bootstrapping) between blocks
"""
