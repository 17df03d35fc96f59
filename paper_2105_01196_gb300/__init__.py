"""EBIC population fitness evaluation on GB300 (sm_103a).

``paper_2105_01196_gb300.ebic`` is the binding to the C-ABI library ``libebic_gb300.so`` built
from ``csrc/``; ``paper_2105_01196_gb300.synth`` draws seeded synthetic inputs.  Importing this
package loads nothing; importing ``ebic`` loads the library and fails loudly when it is missing.
"""
