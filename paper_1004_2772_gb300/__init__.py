"""GB300-native visited-state store: a lockless shared hash table (find-or-put)
and level-synchronous reachability on it, after Laarman, van de Pol and Weber,
"Boosting Multi-Core Reachability Performance with Shared Hash Tables".

The compute path is the CUDA library built from ``csrc/`` (``_build.py``);
``binding`` is its ctypes binding and ``synth`` the seeded input generator.
Nothing here falls back to the CPU.
"""

__all__ = ["binding", "synth"]
