"""GB300-native Count Sketch Kaczmarz (CSK) solver (arXiv 2004.02480)."""
