"""CPU oracle for the HE-LRM hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, independent restatement of what the encrypted DLRM path
computes: RNS-CKKS (HE-LRM appendix "CKKS operations"), hybrid key switching,
Galois rotations, the diagonal / baby-step giant-step matrix-vector product
(Sec. 2.1.4, Sec. 3.2.1) with double hoisting, the client-side digit
decomposition and one-hot selectors (Sec. 4.1), the block-diagonal multi-table
packing (Sec. 4.2.2) and the end-to-end DLRM protocol (Sec. 5.3).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never imports, links or
calls it, and it shares no code, table or constant generator with the library.

Modules:
  ring     -- ctypes loader for ring.c (128-bit modmul, schoolbook convolution,
              textbook NTT), with numpy wrappers.
  primes   -- Miller-Rabin prime search and primitive roots.
  chacha   -- ChaCha20 block function (RFC 8439) and the samplers built on it.
  ckks     -- the scheme: encode/decode, keys, encryption, ring operations,
              rescale, ModUp/ModDown, key switching, rotation.
  linear   -- diagonal layout, BSGS split and the double-hoisted matvec.
  dlrm     -- digit decomposition, selectors, packing, the model compiler,
              the encrypted pipeline and the FP64 cleartext DLRM.
"""
