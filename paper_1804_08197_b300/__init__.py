"""B300-native direct-volume-rendering hot path of syGlass (arXiv:1804.08197).

The product is the C-ABI library ``libsg.so`` (declared in ``include/sg.h``,
built from ``csrc/`` by ``build.py``); ``sg`` is its thin ctypes binding.
"""
