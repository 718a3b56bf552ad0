"""GB300-native fast high-dimensional bilateral and nonlocal-means filtering
(Nair & Chaudhury, arXiv 1811.02363).

``paper_1811_02363_gb300.api``  the Python surface over the CUDA library
                                 (``HDFilter``, ``bruteforce``); importing it
                                 loads ``lib/libhdfilter.so`` and fails if it
                                 has not been built.
``paper_1811_02363_gb300.build`` builds the library with nvcc for sm_103a.
``paper_1811_02363_gb300.synthetic`` seeded synthetic inputs.
"""
